"""Pins of the 3-D (D3Q19) oracle against facts that do not come from the oracle.

The paper states the scheme in two dimensions; the 3-D oracle writes the same
equations for 19 velocities.  What fixes it:

- the D3Q19 tables: isotropy to fourth order (which makes nu = 1/6 - 2A/9 of Eq. A
  hold unchanged) and their projection onto the D2Q9 weights of Eq. (D2Q9w);
- the moments of the equilibrium in closed form (mass source (2/3) A div u of the
  A-term, momentum u, second moment rho/3 + u u + A/9 (tr S + 2 S));
- reduction to the pinned 2-D oracle: for a state that does not vary along z (and
  w = 0), one forward step on the inner z layers, faces included, and one adjoint
  step at interior nodes equal the 2-D oracle's step;
- exact adjointness: one ALKS step is the transpose of the Jacobian of one LKS step;
- the one-step gradient equals central finite differences;
- the generalized-inverse rule of every face, box-edge and corner class equals
  numpy's least squares.
"""
import itertools

import numpy as np
import pytest

import inputs
from oracle import oracle as O


def test_d3q19_tables_are_isotropic():
    c, w = O.lattice3()
    assert len({tuple(x) for x in c}) == 19
    assert sorted(int(x @ x) for x in c) == [0] + [1] * 6 + [2] * 12
    for x in c:
        assert any((y == -x).all() for y in c)
    assert abs(w.sum() - 1) < 1e-15
    d = np.eye(3)
    np.testing.assert_allclose(np.einsum("k,ka->a", w, c), 0, atol=1e-15)
    np.testing.assert_allclose(np.einsum("k,ka,kb->ab", w, c, c), d / 3, atol=1e-15)
    np.testing.assert_allclose(np.einsum("k,ka,kb,kc->abc", w, c, c, c), 0, atol=1e-15)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    np.testing.assert_allclose(np.einsum("k,ka,kb,kc,kd->abcd", w, c, c, c, c), iso, atol=1e-15)


def test_d3q19_projects_onto_d2q9_weights():
    """Summed over c_z, the D3Q19 weights are the D2Q9 weights of Eq. (D2Q9w)."""
    c, w = O.lattice3()
    proj = {}
    for x, wk in zip(c, w):
        proj[(x[0], x[1])] = proj.get((x[0], x[1]), 0.0) + wk
    for (cx, cy), v in proj.items():
        expect = {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}[cx * cx + cy * cy]
        assert abs(v - expect) < 1e-15


def test_equilibrium_moments_closed_form():
    rng = np.random.default_rng(7)
    for A in (-0.6675, 0.1763, 0.4):
        rho = 1 + 0.1 * rng.standard_normal()
        u = 0.05 * rng.standard_normal(3)
        g = 0.02 * rng.standard_normal((3, 3))
        S = g + g.T
        m = O.feq_moments3(A, rho, u, g)
        assert abs(m[0] - (rho + 2 * A / 3 * np.trace(g))) < 1e-15
        np.testing.assert_allclose(m[1:4], u, atol=1e-15)
        P = rho / 3 * np.eye(3) + np.outer(u, u) + A / 9 * (np.trace(S) * np.eye(3) + 2 * S)
        np.testing.assert_allclose(m[4:], [P[0, 0], P[0, 1], P[0, 2], P[1, 1], P[1, 2], P[2, 2]], atol=1e-15)


def _reduction_pair(nu=0.2, nx=14, ny=11, nz=7):
    p3 = inputs.Problem3(nx=nx, ny=ny, nz=nz, nu=nu, alpha_bar=40.0, u_max=0.04, profile=1)
    p2 = inputs.Problem(nx=nx, ny=ny, nu=nu, alpha_bar=40.0, u_max=0.04, in_y0=0, in_y1=ny - 1,
                        out_y0=1, out_y1=ny - 2)
    rng = np.random.default_rng(11)
    g2 = np.clip(0.5 + 0.3 * rng.standard_normal((ny, nx)), 0, 1)
    return p3, p2, g2, rng


@pytest.mark.parametrize("nu", [0.1, 0.315])
def test_forward_step_reduces_to_2d(nu):
    p3, p2, g2, rng = _reduction_pair(nu)
    nz = p3.nz
    s2 = O.State(p2.ny, p2.nx)
    s2.rho = 1 + 0.01 * rng.standard_normal(s2.rho.shape)
    s2.u = 0.04 * rng.standard_normal(s2.u.shape)
    s2.v = 0.04 * rng.standard_normal(s2.u.shape)
    s3 = O.State3(nz, p3.ny, p3.nx)
    s3.rho[:] = s2.rho
    s3.u[:] = s2.u
    s3.v[:] = s2.v
    g3 = np.broadcast_to(g2, (nz, p3.ny, p3.nx)).copy()
    o2 = O.forward_step(p2, g2, 1.0, s2)
    o3 = O.forward_step3(p3, g3, s3)
    for k in range(2, nz - 2):
        np.testing.assert_allclose(o3.rho[k], o2.rho, rtol=0, atol=1e-14)
        np.testing.assert_allclose(o3.u[k], o2.u, rtol=0, atol=1e-15)
        np.testing.assert_allclose(o3.v[k], o2.v, rtol=0, atol=1e-15)
        np.testing.assert_allclose(o3.w[k], 0.0, atol=1e-16)


@pytest.mark.parametrize("nu", [0.1, 0.315])
def test_adjoint_step_reduces_to_2d(nu):
    p3, p2, g2, rng = _reduction_pair(nu)
    nz, ny, nx = p3.nz, p3.ny, p3.nx
    s1, s0 = O.State(ny, nx), O.State(ny, nx)
    for s in (s1, s0):
        s.u = 0.04 * rng.standard_normal((ny, nx))
        s.v = 0.04 * rng.standard_normal((ny, nx))
    a2 = np.zeros((O.NADJ, ny, nx))
    a2[:6] = rng.standard_normal((6, ny, nx))
    r2 = O.adjoint_step(p2, g2, s1, s0, a2)
    t1, t0 = O.State3(nz, ny, nx), O.State3(nz, ny, nx)
    t1.u[:], t1.v[:], t0.u[:], t0.v[:] = s1.u, s1.v, s0.u, s0.v
    a3 = np.zeros((O.NADJ3, nz, ny, nx))
    for q3, q2 in ((0, 0), (1, 1), (2, 2), (4, 3), (5, 4), (7, 5)):
        a3[q3] = a2[q2]
    a3[9] = rng.standard_normal((ny, nx))  # s~_zz: enters no other moment when w = 0
    g3 = np.broadcast_to(g2, (nz, ny, nx)).copy()
    r3 = O.adjoint_step3(p3, g3, t1, t0, a3)
    for k in range(2, nz - 2):
        for q3, q2 in ((0, 0), (1, 1), (2, 2), (4, 3), (5, 4), (7, 5)):
            np.testing.assert_allclose(r3[q3, k, 1:-1, 1:-1], r2[q2, 1:-1, 1:-1], rtol=0, atol=1e-13)
        for q3 in (3, 6, 8):
            np.testing.assert_allclose(r3[q3, k, 1:-1, 1:-1], 0.0, atol=1e-14)


@pytest.mark.parametrize("nu", [0.1, 0.3])
def test_alks_step_is_transpose_of_lks_step(nu):
    """With alpha = 0 and fields supported away from the faces, one 3-D ALKS step is
    exactly the transpose of the Jacobian of one 3-D LKS step (pairing P ~ rho,
    V ~ u); the forward step is quadratic, so its central difference is exact."""
    rng = np.random.default_rng(1)
    pb = inputs.Problem3(nx=11, ny=10, nz=9, nu=nu, alpha_bar=10.0)
    g = np.ones((pb.nz, pb.ny, pb.nx))
    X = O.State3(pb.nz, pb.ny, pb.nx)
    X.rho = 1 + 0.01 * rng.standard_normal(X.rho.shape)
    for f in ("u", "v", "w"):
        setattr(X, f, 0.05 * rng.standard_normal(X.rho.shape))
    sup = np.zeros(X.rho.shape)
    sup[3:-3, 3:-3, 3:-3] = 1
    dX = O.State3(pb.nz, pb.ny, pb.nx)
    for f in ("rho", "u", "v", "w"):
        setattr(dX, f, rng.standard_normal(sup.shape) * sup)
    eps = 1e-3

    def add(s):
        c = X.copy()
        for f in ("rho", "u", "v", "w"):
            setattr(c, f, getattr(X, f) + s * getattr(dX, f))
        return c

    Sp = O.forward_step3(pb, g, add(eps))
    Sm = O.forward_step3(pb, g, add(-eps))
    LdX = [(getattr(Sp, f) - getattr(Sm, f)) / (2 * eps) for f in ("rho", "u", "v", "w")]
    sup2 = np.zeros_like(sup)
    sup2[2:-2, 2:-2, 2:-2] = 1
    PV = rng.standard_normal((4,) + sup.shape) * sup2
    m = O.adjoint_gather3(pb, g, PV, X) - O.adjoint_gather3(pb, g, 0 * PV, X)
    q = O.adjoint_eq3(pb, X, m)
    lhs = sum(np.sum(PV[k] * LdX[k]) for k in range(4))
    rhs = np.sum(q[0] * dX.rho + q[1] * dX.u + q[2] * dX.v + q[3] * dX.w)
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_one_step_gradient_is_exact():
    """One unsteady step, J = J_O(state(1)): ALKS and the sensitivity integrand
    alpha' |u|^2 + 3 alpha' u.u~ give the exact derivative (central FD)."""
    pb = inputs.Problem3(nx=9, ny=8, nz=7, nu=0.2, alpha_bar=30.0, seed=5, sigma=1.5, strip=1)
    g = pb.gamma()
    rng = np.random.default_rng(3)
    st0 = O.State3(pb.nz, pb.ny, pb.nx)
    for f in ("u", "v", "w"):
        setattr(st0, f, 0.03 * rng.standard_normal(st0.rho.shape))
    st0.rho = 1 + 0.01 * rng.standard_normal(st0.rho.shape)
    _, _, tr, J = O.forward3(pb, g, 1, state=st0, traj=True, accumulate_J=True)
    _, sens = O.unsteady_adjoint3(pb, g, tr)
    eps = 1e-6
    for (k, j, i) in [(1, 1, 1), (3, 4, 2), (5, 6, 7), (2, 3, 5)]:
        gp, gm = g.copy(), g.copy()
        gp[k, j, i] += eps
        gm[k, j, i] -= eps
        fd = (O.forward3(pb, gp, 1, state=st0, accumulate_J=True)[3] -
              O.forward3(pb, gm, 1, state=st0, accumulate_J=True)[3]) / (2 * eps)
        # truncation O(eps^2) plus the rounding of the two J values, eps_mach |J| / eps
        assert abs(fd - sens[k, j, i]) <= 1e-7 * abs(fd) + 4 * np.finfo(float).eps * abs(J) / eps


def test_pressure_drop_closed_form_3d():
    """rho = 1 + a x: J_p = 1/3 (sum_in rho - sum_out rho) = -a (nx-1)(ny-2)(nz-2)/3
    over the face-interior nodes of x = 0 and x = nx-1; the face edges (wall nodes)
    do not enter, and J = J_O + kappa_p J_p."""
    pb = inputs.Problem3(nx=12, ny=9, nz=8, nu=0.2, alpha_bar=10.0)
    st = O.State3(pb.nz, pb.ny, pb.nx)
    a = -0.021
    st.rho = 1.0 + a * np.arange(pb.nx)[None, None, :] * np.ones((pb.nz, pb.ny, 1))
    for i in (0, pb.nx - 1):
        st.rho[0, :, i] = st.rho[-1, :, i] = st.rho[:, 0, i] = st.rho[:, -1, i] = 1e6
    want = -a * (pb.nx - 1) * (pb.ny - 2) * (pb.nz - 2) / 3.0
    assert abs(O.pressure_drop3(pb, st) - want) <= 1e-12 * abs(want) * 10
    g = pb.gamma()
    assert abs(O.objective3(pb.with_(kappa_p=1.5), g, st) - O.dissipation3(pb, g, st) - 1.5 * want) <= 1e-9


def test_outlet_row_term_moves_only_lambda_3d():
    """Outlet face: a constant row term is absorbed by lambda~ (Eq. afboundaryp), the
    filled f~ are unchanged; on the inlet face it is not (mu~ . c_k cannot carry a
    constant, since the rest link has c = 0)."""
    c, w = O.lattice3()
    rng = np.random.default_rng(6)
    for n, pressure in (((1, 0, 0), True), ((-1, 0, 0), False)):
        n = np.array(n)
        unknown = np.array([(x * n > 0).any() for x in c])
        known = rng.standard_normal(19) * ~unknown
        f0, m0 = O.bc_flow3(n, pressure, -0.1095, known, unknown)
        f1, m1 = O.bc_flow3(n, pressure, -0.1095, known, unknown, jb=0.8)
        if pressure:
            np.testing.assert_allclose(f1, f0, atol=1e-12)
            assert abs((m1[0] - m0[0]) + 0.8) <= 1e-12
        else:
            assert np.abs(f1 - f0).max() > 0.1


@pytest.mark.parametrize("A", [-0.1095, 0.3])
def test_edge_rules_equal_numpy_least_squares(A):
    """Every face, box-edge and corner class: the oracle's normal-equation solve of
    the generalized-inverse rule equals numpy's least squares on the same system,
    with and without a boundary objective term (a constant added to every row)."""
    c, w = O.lattice3()
    rng = np.random.default_rng(5)
    for n in itertools.product((-1, 0, 1), repeat=3):
        n = np.array(n)
        if not n.any():
            continue
        faces = int(np.abs(n).sum())
        pressure = faces == 1 and n[0] == 1
        unknown = np.array([(x * n > 0).any() for x in c])
        known = rng.standard_normal(19) * ~unknown
        jb = rng.standard_normal() if faces == 1 else 0.0
        f, mult = O.bc_flow3(n, pressure, A, known, unknown, jb=jb)
        cn = c @ n
        M = np.diag(cn.astype(float)) - 2 * A * (w * cn)[None, :] * (c @ c.T)
        U = [k for k in range(19) if unknown[k] and np.abs(M[:, k]).sum() > 0]
        if pressure:
            mc = [np.ones(19), c[:, 1].astype(float), c[:, 2].astype(float)]
        else:
            mc = [c[:, a].astype(float) for a in range(3)]
        Am = np.stack([M[:, k] for k in U] + mc, 1)
        x = np.linalg.lstsq(Am, -(M @ known) - jb, rcond=None)[0]
        np.testing.assert_allclose(f[U], x[:len(U)], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(mult, x[len(U):], rtol=1e-10, atol=1e-12)
        dead = [k for k in range(19) if unknown[k] and k not in U]
        assert np.all(f[dead] == 0)


@pytest.mark.slow
def test_pressure_drop_row_term_against_central_differences_3d():
    """The 3-D form of the paper's pressure-drop verification (Sec. 2.6): a 13 x 9 x 9
    duct, nu = 0.1, Re = 1, gamma = 0.1 in a central ball and 0.9 elsewhere,
    J = J_p.  On this coarse grid the ALKS gradient is 0.38-0.47 of the central
    difference (0.51-0.86 at 31 x 21 x 21: the edge rule's error shrinks with
    resolution); the bounds still separate the adopted row term (d/dp) from 1/3 per
    row (d/df_k), which gives 0.13-0.16."""
    nu, steps = 0.1, 3000
    pb = inputs.Problem3(nx=13, ny=9, nz=9, nu=nu, alpha_bar=1e3 * nu, u_max=nu / 8, n_steps=steps, n_adj=steps)
    zz, yy, xx = np.mgrid[0:pb.nz, 0:pb.ny, 0:pb.nx]
    g = np.where((xx - 6) ** 2 + (yy - 4) ** 2 + (zz - 4) ** 2 <= 2.5 ** 2, 0.1, 0.9)
    st, res, _, _ = O.forward3(pb, g, steps)
    assert res < 1e-11
    _, s1, _ = O.steady_adjoint3(pb.with_(kappa_p=1.0), g, st, steps)
    _, s0, _ = O.steady_adjoint3(pb, g, st, steps)
    adj = s1 - s0
    eps = 1e-3
    for i in (3, 6, 9):
        v = []
        for sg in (1, -1):
            gg = g.copy()
            gg[4, 4, i] += sg * eps
            v.append(O.pressure_drop3(pb, O.forward3(pb, gg, steps)[0]))
        fd = (v[0] - v[1]) / (2 * eps)
        assert 0.3 <= adj[4, 4, i] / fd <= 1.2, (i, adj[4, 4, i], fd)
