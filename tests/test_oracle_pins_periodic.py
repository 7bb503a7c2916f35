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


# --------------------------------------------------------------------------------------
# Heat source (Eqs. heatsource, betagamma) and Boussinesq force (Eq. boussinesqforce)
# --------------------------------------------------------------------------------------
def beta_paper(beta_bar, q, g):
    """Eq. (betagamma): beta_gamma = beta_bar q (1 - gamma) / (q + gamma)."""
    return beta_bar * q * (1.0 - g) / (q + g)


@pytest.mark.parametrize("g0", [0.0, 0.4])
def test_heat_source_relaxation_closed_form(g0):
    """Fluid at rest with uniform T on a periodic box: the thermal step maps T to
    (T + beta_gamma) / (1 + beta_gamma) (source Q = beta_gamma (1 - T) of Eq.
    heatsource at t + dt, Eq. lbeg_ex), so T_n = 1 - (1 - T_0)(1 + beta)^-n: the
    solid heats towards 1.  gamma = 0 gives beta = beta_bar for any q_beta."""
    bb, q = 0.3, 0.1
    pb = inputs.Problem(nx=6, ny=5, nu=0.1, alpha_bar=0.0, u_max=0.0, periodic=3, thermal=1, K_f=0.1, K_s=0.1,
                        beta_bar=bb, q_beta=q)
    g = np.full((pb.ny, pb.nx), g0)
    b = beta_paper(bb, q, g0)
    st = O.State(pb.ny, pb.nx)
    st.T[:] = 0.2
    done = 0
    for n in (1, 3, 25):
        st, _, _, _ = O.forward(pb, g, n - done, state=st)
        done = n
        assert np.abs(st.T - (1.0 - 0.8 * (1.0 + b) ** (-n))).max() <= 1e-14
        assert np.abs(st.u).max() == 0.0


def test_boussinesq_force_of_a_uniform_temperature():
    """Uniform T != T_ref on a periodic box: G = g beta (T - T_ref) is uniform, so the
    velocity follows the implicit Darcy march u_n = (G / alpha)(1 - (1 + alpha)^-n)
    (Eq. lbef_ex with Eq. boussinesqforce); T stays uniform."""
    pb = inputs.Problem(nx=6, ny=5, nu=0.1, alpha_bar=2.0, q_alpha=0.1, u_max=0.0, periodic=3, thermal=1,
                        K_f=0.1, K_s=0.1, gb_x=2e-4, gb_y=-7e-4, T_ref=0.25)
    g = np.full((pb.ny, pb.nx), 0.3)
    a = alpha_paper(2.0, 0.1, 0.3)
    st = O.State(pb.ny, pb.nx)
    st.T[:] = 0.75
    st, _, _, _ = O.forward(pb, g, 9, state=st)
    for comp, gb in (("u", pb.gb_x), ("v", pb.gb_y)):
        G = gb * (0.75 - 0.25)
        assert np.abs(getattr(st, comp) - G / a * (1 - (1 + a) ** -9)).max() <= 1e-15 * 9 + 1e-13 * abs(G / a)
    assert np.abs(st.T - 0.75).max() <= 1e-14


def test_one_step_gradient_with_heat_source_and_boussinesq_is_exact():
    """Unsteady thermal problem of one step, J = J_O(state(1)) with the dissipation,
    kappa_T sum T and the heat-exchange objective -kappa_Q sum beta_gamma (1 - T)
    (Eq. objective_heatexchanger), a heat source and a Boussinesq force: the ALKS
    level-1 adjoint (T~ with the implicit source division and the 3 g beta . u~
    coupling of Eq. albeg_ex) and the sensitivity terms 3 alpha' u.u~,
    -beta' (1 - T) T~ and -kappa_Q beta' (1 - T) give the exact derivative, compared
    with central differences.  K_s = K_f, so the B-term (level 0) is absent."""
    pb = inputs.Problem(nx=12, ny=10, nu=0.2, alpha_bar=30.0, seed=4, sigma=1.5, strip=1, steady=False, n_steps=1,
                        thermal=1, K_f=0.1, K_s=0.1, kappa_T=0.3, beta_bar=0.2, q_beta=0.1, kappa_Q=0.7,
                        gb_x=0.01, gb_y=-0.02, T_ref=0.4, t_kind=[0, 1, 0, 1], t_val=[0.0, 0.0, 1.0, 0.0])
    g = pb.gamma()
    rng = np.random.default_rng(3)
    st0 = O.State(pb.ny, pb.nx)
    st0.u = 0.03 * rng.standard_normal(st0.u.shape)
    st0.v = 0.03 * rng.standard_normal(st0.u.shape)
    st0.rho = 1 + 0.01 * rng.standard_normal(st0.u.shape)
    st0.T = rng.random(st0.u.shape)
    _, _, tr, J = O.forward(pb, g, 1, state=st0, traj=True, accumulate_J=True)
    adj, sens = O.unsteady_adjoint(pb, g, tr)
    # J ~ 10 (the kappa_T sum T term), so the step is 1e-4: the central difference
    # error then falls as eps^2 (3.6e-5 at 1e-3, 3.6e-7 at 1e-4) down to round-off
    eps = 1e-4
    for (j, i) in [(1, 1), (3, 4), (5, 7), (8, 10), (4, 2)]:
        gp, gm = g.copy(), g.copy()
        gp[j, i] += eps
        gm[j, i] -= eps
        Jp = O.forward(pb, gp, 1, state=st0, accumulate_J=True)[3]
        Jm = O.forward(pb, gm, 1, state=st0, accumulate_J=True)[3]
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - sens[j, i]) <= 1e-6 * abs(fd), (j, i, fd, sens[j, i])


# --------------------------------------------------------------------------------------
# Natural convection: the paper's sensitivity check (Sec. 2.6) on a closed cavity
# --------------------------------------------------------------------------------------
@pytest.mark.slow
def test_natural_convection_cavity_alks_agrees_with_central_differences():
    """Sec. 2.6's natural-convection check at half resolution (70 x 40 dx): closed
    cavity, T = 0 on the left, right and top walls, adiabatic bottom with a heated
    centre part (heat flux), Boussinesq force (Ra = 2e4, Pr = 0.71), K_s = 10 K_f,
    gamma = 0.1 in the central 20 x 13 block and 0.9 around it, J = kappa_T sum T.
    On the converged state the ALKS sensitivity and central differences (eps = 1e-3)
    along the centre line agree in direction (cosine >= 0.99); their ratio is 1.3-1.4
    inside the gamma = 0.1 block and 2.7-3.2 in the gamma = 0.9 ring, the continuous
    adjoint's error at the coefficient jumps that the paper also reports."""
    pb, g = inputs.natural_convection_cavity(0.5)
    st, res, _ = O.forward_to_steady(pb, g, tol=1e-13, max_steps=300000, chunk=2000)
    assert res < 1e-12
    _, sens, ares = O.steady_adjoint(pb, g, st, 40000)
    assert ares < 1e-6
    j, eps = pb.ny // 2, 1e-3
    a, b = [], []
    for i in (20, 28, 36, 44, 52):
        v = []
        for sg in (1, -1):
            gg = g.copy()
            gg[j, i] += sg * eps
            s2, _, _ = O.forward_to_steady(pb, gg, tol=1e-13, max_steps=300000, chunk=1000, state=st)
            v.append(O.objective(pb, gg, s2))
        a.append(sens[j, i])
        b.append((v[0] - v[1]) / (2 * eps))
    a, b = np.array(a), np.array(b)
    assert a @ b / np.linalg.norm(a) / np.linalg.norm(b) >= 0.99
    assert np.all((a / b > 1.0) & (a / b < 4.0)), a / b


# --------------------------------------------------------------------------------------
# Forced convection with the heat source: the paper's second sensitivity check (Sec. 2.6)
# --------------------------------------------------------------------------------------
@pytest.mark.slow
def test_forced_convection_check_alks_agrees_with_central_differences():
    """Sec. 2.6's forced-convection check on the 31 x 31 domain of its non-thermal
    check (inputs.forced_convection_check): T = 0 on the inlet edge, adiabatic
    elsewhere, the solid heating the fluid through Q = beta_gamma (1 - T), and the
    heat-exchange objective.  Its sensitivity (kappa_Q = 1 minus kappa_Q = 0, the
    dissipation's share removed) agrees with central differences (eps = 1e-3) of the
    heat-exchange objective along the centre line: cosine >= 0.999 and ratios within
    0.8..1.05 at Pr = 0.71 (0.82 at the node nearest the outlet, 0.92..0.97 elsewhere).  At Pr = 6 (a tenth of the diffusivity) the direction
    still agrees but the ratios spread to 0.3..0.8, the continuous adjoint's boundary
    and advection error that the paper reports for this check."""
    pb, g = inputs.forced_convection_check()
    st, res, _ = O.forward_to_steady(pb, g, tol=1e-14, max_steps=400000, chunk=2000)
    assert res < 1e-13
    _, s1, r1 = O.steady_adjoint(pb, g, st, 60000)
    _, s0, _ = O.steady_adjoint(pb.with_(kappa_Q=0.0), g, st, 60000)
    assert r1 < 1e-10
    sens = s1 - s0
    assert np.abs(sens).max() > 0

    def JQ(gg, s):
        return O.objective(pb, gg, s) - O.objective(pb.with_(kappa_Q=0.0), gg, s)

    eps, j = 1e-3, 15
    a, b = [], []
    for i in (6, 10, 15, 21, 25):
        v = []
        for sg in (1, -1):
            gg = g.copy()
            gg[j, i] += sg * eps
            s2, _, _ = O.forward_to_steady(pb, gg, tol=1e-14, max_steps=400000, chunk=1000, state=st)
            v.append(JQ(gg, s2))
        a.append(sens[j, i])
        b.append((v[0] - v[1]) / (2 * eps))
    a, b = np.array(a), np.array(b)
    assert a @ b / np.linalg.norm(a) / np.linalg.norm(b) >= 0.999
    assert np.all((a / b > 0.8) & (a / b < 1.05)), a / b
