"""Pins of the FP64 CPU oracle on periodic lattices and on prescribed fields.

These fix the parts of the oracle that the channel pins leave open:

- the Brinkman interpolation alpha_gamma (Eq. brinkman) together with the implicit
  Brinkman update u = (u* + G) / (1 + alpha_gamma) of Eq. (lbef_ex);
- the value of the dissipation objective J_O (not only its derivative);
- the relation between nu and A (Eq. A) away from walls;
- the conservation of mass and momentum by the interior stencil.

Each test compares the oracle with a closed form or an exact identity of the
discrete scheme.  Periodic axes and the uniform force G exist in the oracle only;
the CUDA path rejects them.
"""
import os

import numpy as np
import pytest

os.environ.setdefault("OMP_NUM_THREADS", "2")

import inputs  # noqa: E402
from oracle import oracle as O  # noqa: E402


def alpha_paper(alpha_bar, q, g):
    """Eq. (brinkman): alpha_gamma = alpha_bar q (1 - gamma) / (q + gamma)."""
    return alpha_bar * q * (1.0 - g) / (q + g)


# --------------------------------------------------------------------------------------
# Darcy limit: uniform design, uniform force, fully periodic box
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("g0", [0.0, 0.3, 0.85])
def test_darcy_limit_implicit_brinkman(g0):
    """Uniform fields have no gradients, so one LKS step maps u to
    (u + G) / (1 + alpha_gamma) exactly (first moment of f^eq is u; the Brinkman
    term of Eq. lbef_ex taken at t + dt).  From rest the march is
    u_n = (G / alpha)(1 - (1 + alpha)^-n), which tends to Darcy's u = G / alpha.
    An explicit Brinkman term would give u_1 = G; a misplaced q_alpha changes alpha.
    gamma = 0 checks alpha = alpha_bar (solid), independently of q_alpha."""
    ab, q = 2.0, 0.1
    pb = inputs.Problem(nx=6, ny=5, nu=0.1, alpha_bar=ab, q_alpha=q, u_max=0.0, periodic=3,
                        G_x=1e-4, G_y=-3e-5)
    g = np.full((pb.ny, pb.nx), g0)
    a = alpha_paper(ab, q, g0)
    if g0 == 0.0:
        assert a == ab
    st = O.State(pb.ny, pb.nx)
    done = 0
    for n in (1, 2, 7, 40):
        st, _, _, _ = O.forward(pb, g, n - done, state=st)
        done = n
        for comp, G in (("u", pb.G_x), ("v", pb.G_y)):
            expect = G / a * (1.0 - (1.0 + a) ** (-n))
            got = getattr(st, comp)
            # round-off of sums of O(1) populations, accumulated over n steps
            assert np.abs(got - expect).max() <= 1e-15 * n + 1e-13 * abs(G / a), (n, comp)
        assert np.abs(st.rho - 1.0).max() <= 1e-15 * n


# --------------------------------------------------------------------------------------
# Brinkman-Stokes channel: periodic in x, node walls at y = 0 and y = H
# --------------------------------------------------------------------------------------
def _brinkman_channel(H, kH=4.0, nu=0.1, ab=100.0, q=0.1, umax=0.01):
    """Converged oracle state of the periodic channel with a uniform design whose
    alpha_gamma keeps k H fixed (k^2 = alpha / nu), driven by a uniform force."""
    alpha = nu * (kH / H) ** 2
    g0 = q * (ab - alpha) / (alpha + ab * q)          # inverse of Eq. (brinkman)
    assert abs(alpha_paper(ab, q, g0) - alpha) < 1e-15 * ab
    G = umax * alpha / (1.0 - 1.0 / np.cosh(kH / 2))
    pb = inputs.Problem(nx=5, ny=H + 1, nu=nu, alpha_bar=ab, q_alpha=q, u_max=0.0, periodic=1, G_x=G)
    g = np.full((pb.ny, pb.nx), g0)
    st, res, _ = O.forward_to_steady(pb, g, tol=1e-14 * umax, max_steps=200000, chunk=2000)
    assert res < 1e-14 * umax
    y = np.arange(H + 1)
    k = kH / H
    exact = (G / alpha) * (1.0 - np.cosh(k * (y - H / 2)) / np.cosh(k * H / 2))
    return st, exact, umax


def test_brinkman_stokes_channel_converges_second_order():
    """Fully developed flow through a uniform porous channel: nu u'' - alpha u + G = 0
    with u = 0 on the walls (the steady form of Eq. ns with the Brinkman and force
    terms), u = (G/alpha)(1 - cosh(k(y - H/2)) / cosh(kH/2)), k = sqrt(alpha / nu).
    With k H fixed the oracle's steady profile converges to it at second order:
    the maximum error falls by about 4 for each doubling of H (observed 5.1 and 4.6,
    approaching 4 from above), and v = 0, uniform in x.  A first-order error would
    fall by 2; a wrong alpha, force or Brinkman division leaves an O(1) error."""
    errs = []
    for H in (8, 16, 32):
        st, exact, umax = _brinkman_channel(H)
        assert np.abs(st.v).max() <= 1e-13 * umax
        assert np.abs(st.u - st.u[:, :1]).max() <= 1e-13 * umax
        errs.append(np.abs(st.u[:, 0] - exact).max() / umax)
    assert errs[0] < 0.05
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.5 < e0 / e1 < 5.5, errs


def test_brinkman_stokes_channel_dissipation():
    """J_O of the converged Brinkman channel equals the closed form
    sum over interior nodes of nu (du/dy)^2 + alpha u^2 (dissipation of Eq. fj with
    S_xy = du/dy the only strain), evaluated on the exact profile, to the scheme's
    O(h^2) accuracy; with the exact profile fed in it matches to round-off up to the
    central-difference error of du/dy."""
    H = 32
    st, exact, umax = _brinkman_channel(H)
    pb = inputs.Problem(nx=5, ny=H + 1, nu=0.1, alpha_bar=100.0, q_alpha=0.1, u_max=0.0, periodic=1)
    alpha = 0.1 * (4.0 / H) ** 2
    g0 = 0.1 * (100.0 - alpha) / (alpha + 100.0 * 0.1)
    g = np.full((pb.ny, pb.nx), g0)
    J = O.objective(pb, g, st)
    y = np.arange(H + 1)
    k = 4.0 / H
    G = umax * alpha / (1.0 - 1.0 / np.cosh(2.0))
    dudy = -(G / alpha) * k * np.sinh(k * (y - H / 2)) / np.cosh(k * H / 2)
    inner = slice(1, H)
    Jexact = pb.nx * np.sum(pb.nu * dudy[inner] ** 2 + alpha * exact[inner] ** 2)
    assert abs(J / Jexact - 1.0) < 5e-3


# --------------------------------------------------------------------------------------
# The dissipation objective on prescribed fields
# --------------------------------------------------------------------------------------
def _quadratic_fields(nx, ny, rng):
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    cu = rng.standard_normal(6) * np.array([1e-2, 1e-3, 1e-3, 1e-5, 1e-5, 1e-5])
    cv = rng.standard_normal(6) * np.array([1e-2, 1e-3, 1e-3, 1e-5, 1e-5, 1e-5])

    def val(c):
        return c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y

    def dx(c):
        return c[1] + 2 * c[3] * x + c[4] * y

    def dy(c):
        return c[2] + c[4] * x + 2 * c[5] * y

    return val(cu), val(cv), dx(cu), dy(cu), dx(cv), dy(cv)


@pytest.mark.parametrize("gval", [1.0, 0.0])
def test_dissipation_objective_closed_form(gval):
    """J_O = sum over interior nodes of nu/2 (S_xx^2 + 2 S_xy^2 + S_yy^2)
    + alpha_gamma |u|^2 + kappa_T T with S_ab = du_a/dx_b + du_b/dx_a, on quadratic
    u, v fields whose derivatives are written out analytically (central differences
    are exact on quadratics).  gamma = 1 (alpha = 0) isolates the strain terms; gamma = 0
    (alpha = alpha_bar, Eq. brinkman) adds the Brinkman term.  A halved S_xy term, nu
    in place of nu/2, or a wrong alpha fails."""
    rng = np.random.default_rng(41)
    nx, ny = 11, 9
    pb = inputs.Problem(nx=nx, ny=ny, nu=0.13, alpha_bar=7.0, thermal=1, K_f=0.1, K_s=0.1, kappa_T=0.37)
    u, v, ux, uy, vx, vy = _quadratic_fields(nx, ny, rng)
    st = O.State(ny, nx)
    st.u, st.v = u.copy(), v.copy()
    st.T = rng.standard_normal((ny, nx))
    g = np.full((ny, nx), gval)
    alpha = 7.0 if gval == 0.0 else 0.0
    Sxx, Syy, Sxy = 2 * ux, 2 * vy, uy + vx
    dens = 0.5 * pb.nu * (Sxx ** 2 + 2 * Sxy ** 2 + Syy ** 2) + alpha * (u ** 2 + v ** 2) + pb.kappa_T * st.T
    expect = dens[1:-1, 1:-1].sum()
    J = O.objective(pb, g, st)
    assert abs(J - expect) <= 1e-13 * np.abs(dens[1:-1, 1:-1]).sum()


def test_poiseuille_dissipation_closed_form():
    """On the converged Poiseuille state of an empty channel (gamma = 1, alpha = 0)
    the only strain is S_xy = du/dy = 4 u_max (H - 2y) / H^2, so
    J_O = (nx - 2) sum_{y=1}^{H-1} nu S_xy(y)^2 (nu/2 times 2 S_xy^2 per node)."""
    nu, umax = 0.1, 0.02
    pb = inputs.poiseuille(33, 17, nu=nu, u_max=umax)
    g = np.ones((pb.ny, pb.nx))
    st, res, _ = O.forward_to_steady(pb, g, tol=1e-14, max_steps=60000, chunk=1000)
    assert res < 1e-13
    H = pb.ny - 1
    y = np.arange(1, H)
    Sxy = 4 * umax * (H - 2 * y) / H ** 2
    expect = (pb.nx - 2) * np.sum(nu * Sxy ** 2)
    assert abs(O.objective(pb, g, st) / expect - 1.0) < 1e-9


# --------------------------------------------------------------------------------------
# Taylor-Green decay: the nu-A relation (Eq. A) on a periodic box
# --------------------------------------------------------------------------------------
def _tg_rate(N, nu, U=1e-5, t0=20, T=200):
    """Measured decay rate of a Taylor-Green vortex of wavenumber k = 2 pi / N."""
    k = 2 * np.pi / N
    pb = inputs.Problem(nx=N, ny=N, nu=nu, alpha_bar=0.0, u_max=0.0, periodic=3)
    g = np.ones((N, N))
    y, x = np.mgrid[0:N, 0:N].astype(float)
    mode_u = -np.cos(k * x) * np.sin(k * y)
    mode_v = np.sin(k * x) * np.cos(k * y)
    st = O.State(N, N)
    st.u = U * mode_u
    st.v = U * mode_v
    st.rho = 1.0 - 0.75 * U * U * (np.cos(2 * k * x) + np.cos(2 * k * y))
    norm = np.sum(mode_u ** 2 + mode_v ** 2)

    def amp(s):
        return np.sum(s.u * mode_u + s.v * mode_v) / norm

    st, _, _, _ = O.forward(pb, g, t0, state=st)
    a0 = amp(st)
    st, _, _, _ = O.forward(pb, g, T, state=st)
    a1 = amp(st)
    return -np.log(a1 / a0) / T, 2 * nu * k * k


@pytest.mark.parametrize("nu", [0.05, 0.25])
def test_taylor_green_decay_matches_nu(nu):
    """A Taylor-Green vortex decays as exp(-2 nu k^2 t) (Eq. ns at small Re).  The
    oracle's rate, with A from Eq. (A) (A > 0 for nu = 0.05, A < 0 for nu = 0.25),
    approaches 2 nu k^2 with an error that falls by about 4 per doubling of N."""
    errs = []
    for N in (16, 32, 64):
        rate, exact = _tg_rate(N, nu)
        errs.append(abs(rate / exact - 1.0))
    assert errs[-1] < 1e-2, errs
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.3 < e0 / e1 < 4.7, errs


# --------------------------------------------------------------------------------------
# Conservation on a periodic box
# --------------------------------------------------------------------------------------
def test_periodic_conservation_of_mass_and_momentum():
    """Without Brinkman term and force, sum rho and sum u are invariants of every LKS
    step on a periodic box: the A-term adds (2/3) A div u to sum_k f^eq, which sums to
    zero under central differences, and sum_k w_k c_k (c.c terms) vanishes.  With a
    uniform alpha and force, sum u maps to (sum u + N G) / (1 + alpha) exactly."""
    rng = np.random.default_rng(8)
    N = 12
    base = dict(nx=N, ny=N - 2, nu=0.2, u_max=0.0, periodic=3)
    st = O.State(N - 2, N)
    st.u = 0.02 * rng.standard_normal((N - 2, N))
    st.v = 0.02 * rng.standard_normal((N - 2, N))
    st.rho = 1.0 + 0.01 * rng.standard_normal((N - 2, N))
    pb = inputs.Problem(alpha_bar=0.0, **base)
    g = np.ones((N - 2, N))
    s = st
    for _ in range(5):
        s1 = O.forward_step(pb, g, 1.0, s)
        assert abs(s1.rho.sum() - s.rho.sum()) <= 1e-12
        assert abs(s1.u.sum() - s.u.sum()) <= 1e-14
        assert abs(s1.v.sum() - s.v.sum()) <= 1e-14
        assert np.abs(s1.u - s.u).max() > 1e-6          # the fields do change
        s = s1
    pb2 = inputs.Problem(alpha_bar=3.0, G_x=2e-4, G_y=5e-5, **base)
    g2 = np.full((N - 2, N), 0.4)
    a = alpha_paper(3.0, pb2.q_alpha, 0.4)
    s1 = O.forward_step(pb2, g2, 1.0, st)
    n = st.u.size
    assert abs(s1.u.sum() - (st.u.sum() + n * pb2.G_x) / (1 + a)) <= 1e-14
    assert abs(s1.v.sum() - (st.v.sum() + n * pb2.G_y) / (1 + a)) <= 1e-14
