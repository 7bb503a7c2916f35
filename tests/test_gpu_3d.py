"""GPU parity of the three-dimensional (D3Q19) steady duct path against the FP64
oracle (``oracle/lks3d_oracle.c``), through the C ABI.

Small ducts cover ragged tiles in x and y (37 = 32 + 5, 44 = 32 + 12, 21 = 2 x 8 + 5;
nx % 4 == 0 runs the TMA-staged FP32 kernels, 37 the plain ones) and a
z-march split over two chunks (nz = 40 = 32 + 8); the FP64 instance matches the
oracle to rounding, the FP32 instance to the FP32 tolerances.  At config 4's full
size (192^3) three forward steps and two adjoint iterations are checked against
the oracle's over the whole lattice and at sampled nodes (interior, faces, box
edges, corners).
"""
import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_2411_03090_gb300 import LKS  # noqa: E402


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def duct(nx=37, ny=21, nz=40, Re=20.0, n=60, **kw):
    return inputs.duct(nx, ny, nz, Re=Re, seed=7, sigma=2.0, strip=2, n_steps=n, n_adj=n, **kw)


def to_state(fields):
    d, u, v, w = [f.double().cpu().numpy() for f in fields]
    s = O.State3(*d.shape)
    s.rho, s.u, s.v, s.w = d + 1.0, u, v, w
    return s


@pytest.mark.parametrize("path", ["auto", "step"])
@pytest.mark.parametrize("real,tol_f,tol_g,tol_J", [("f64", 1e-10, 1e-10, 1e-11), ("f32", 1e-5, 1e-3, 1e-5)])
@pytest.mark.parametrize("shape", [(37, 21, 40), (24, 16, 11), (44, 21, 40)])
def test_gradient_matches_oracle(real, tol_f, tol_g, tol_J, shape, path):
    pb = duct(*shape)
    g = pb.gamma()
    ref = O.steady_gradient3(pb, g)
    s = LKS(pb, real=real, path=path)
    J, grad = s.gradient(torch.from_numpy(g))
    tma = real == "f32" and shape[0] % 4 == 0
    assert s.query().fwd_path == (3 if tma and path == "auto" else 1)
    assert s.query().adj_path == (3 if tma and path == "auto" else 1)
    st = to_state(s.get_state())
    for name in ("u", "v", "w"):
        assert rel_l2(getattr(st, name), getattr(ref["state"], name)) <= tol_f, name
    assert rel_l2(st.rho - 1, ref["state"].rho - 1) <= tol_f * 10
    assert abs(J.item() - ref["J"]) <= tol_J * abs(ref["J"])
    adj = [a.double().cpu().numpy() for a in s.get_adjoint()]
    for q in range(O.NADJ3):
        assert rel_l2(adj[q], ref["adjoint"][q]) <= tol_g, O.ADJ3_NAMES[q]
    gr = grad.double().cpu().numpy()
    assert rel_l2(gr, ref["dJdgamma"]) <= tol_g
    assert np.all(gr[0] == 0) and np.all(gr[:, 0] == 0) and np.all(gr[:, :, 0] == 0)


@pytest.mark.parametrize("shape", [(60, 17, 37), (28, 8, 5), (44, 21, 40), (88, 9, 70), (116, 40, 37), (8, 5, 5),
                                   (12, 6, 23)])
def test_column_kernels_match_step_kernels_and_oracle(shape):
    """The warp-column z-march forward and adjoint (28 x 8 tiles, ragged in x, y and
    z) against the plane-march kernels and the oracle's gradient after the same
    steps.  116 x 40 has tiles whose threads are all off the x and y faces (the fast
    variants)."""
    pb = duct(*shape, n=40, kappa_p=1.0, Re=20.0 if shape[1] >= 9 else 2.0)  # nu >= 0.02
    g = pb.gamma()
    gt = torch.from_numpy(g)
    ref = O.steady_gradient3(pb, g)
    st, adj, gr = {}, {}, {}
    for path in ("column", "step"):
        s = LKS(pb, real="f32", path=path)
        _, grad = s.gradient(gt)
        q = s.query()
        assert (q.fwd_path, q.adj_path) == ((3, 3) if path == "column" else (1, 1))
        assert q.device_status == 0
        st[path] = [f.double().cpu().numpy() for f in s.get_state()]
        adj[path] = [a.double().cpu().numpy() for a in s.get_adjoint()]
        gr[path] = grad.double().cpu().numpy()
    scale = max(np.abs(st["step"][1]).max(), 1e-30)
    for c in range(4):
        assert np.abs(st["column"][c] - st["step"][c]).max() <= 1e-6 * (1.0 if c == 0 else scale), c
    for q in range(O.NADJ3):
        aq = max(np.abs(adj["step"][q]).max(), 1e-30)
        assert np.abs(adj["column"][q] - adj["step"][q]).max() <= 1e-5 * aq, O.ADJ3_NAMES[q]
        assert rel_l2(adj["column"][q], ref["adjoint"][q]) <= 1e-3, O.ADJ3_NAMES[q]
    assert rel_l2(gr["column"], gr["step"]) <= 1e-5
    assert rel_l2(gr["column"], ref["dJdgamma"]) <= 1e-3
    col = to_state([torch.from_numpy(x) for x in st["column"]])
    for name in ("u", "v", "w"):
        assert rel_l2(getattr(col, name), getattr(ref["state"], name)) <= 1e-5, name
    assert rel_l2(col.rho - 1, ref["state"].rho - 1) <= 1e-4


@pytest.mark.parametrize("path", ["auto", "step"])
@pytest.mark.parametrize("real,tol_g,tol_J", [("f64", 1e-10, 1e-11), ("f32", 1e-3, 1e-5)])
@pytest.mark.parametrize("shape", [(44, 21, 40), (37, 21, 40)])
def test_pressure_drop_objective_matches_oracle(real, tol_g, tol_J, shape, path):
    """J = J_O + kappa_p J_p (Eq. objective_pipebend): J, the adjoint (whose inlet and
    outlet edge rules carry the boundary objective term) and dJ/dgamma against the
    oracle; the pressure-drop part alone (kappa_p = 2 minus kappa_p = 0) as well."""
    base = duct(*shape)
    g = base.gamma()
    out = {}
    for kp in (0.0, 2.0):
        pb = base.with_(kappa_p=kp)
        ref = O.steady_gradient3(pb, g)
        s = LKS(pb, real=real, path=path)
        J, grad = s.gradient(torch.from_numpy(g))
        assert abs(J.item() - ref["J"]) <= tol_J * abs(ref["J"])
        adj = [a.double().cpu().numpy() for a in s.get_adjoint()]
        for q in range(O.NADJ3):
            assert rel_l2(adj[q], ref["adjoint"][q]) <= tol_g, (kp, O.ADJ3_NAMES[q])
        out[kp] = (J.item(), grad.double().cpu().numpy(), ref)
    Jp = out[2.0][0] - out[0.0][0]
    Jp_ref = out[2.0][2]["J"] - out[0.0][2]["J"]
    assert abs(Jp - Jp_ref) <= 10 * tol_J * abs(out[2.0][2]["J"])
    dg = out[2.0][1] - out[0.0][1]
    dg_ref = out[2.0][2]["dJdgamma"] - out[0.0][2]["dJdgamma"]
    assert rel_l2(dg, dg_ref) <= 3 * tol_g


def test_gradient_host_and_query():
    pb = duct(24, 16, 11, n=20)
    g = pb.gamma()
    s = LKS(pb, real="f32")
    J, grad = s.gradient(torch.from_numpy(g))
    Jh, gh = s.gradient_host(g.astype(np.float32))
    assert Jh == J.item()
    np.testing.assert_array_equal(gh, grad.cpu().numpy())
    q = s.query()
    assert q.device_status == 0 and q.forward_steps == 40 and q.adjoint_steps == 40


def _sample_nodes(pb, rng, n_interior=40):
    nx, ny, nz = pb.nx, pb.ny, pb.nz
    nodes = {(0, 0, 0), (nx - 1, ny - 1, nz - 1), (0, ny // 2, nz // 2), (nx - 1, ny // 3, nz // 2),
             (nx // 2, 0, nz // 2), (nx // 2, ny - 1, 7), (nx // 3, ny // 2, 0), (5, 9, nz - 1),
             (0, 0, nz // 2), (nx - 1, 0, 5), (nx // 2, 0, 0), (33, ny - 1, nz - 1), (1, 1, 1),
             (nx - 2, ny - 2, nz - 2), (31, 7, 31), (32, 8, 32), (63, 15, 95), (64, 16, 96)}
    for _ in range(n_interior):
        nodes.add(tuple(int(rng.integers(0, m)) for m in (nx, ny, nz)))
    return sorted(nodes)


@pytest.fixture(scope="module")
def config4_oracle_short():
    """The oracle's config-4 duct (192^3) after 3 forward steps from rest and 2 adjoint
    iterations on that state (FP64; a few seconds on the host cores)."""
    pb = inputs.config4().with_(n_steps=3, n_adj=2)
    g = pb.gamma()
    st, _, _, _ = O.forward3(pb, g, 3)
    adj, _, _ = O.steady_adjoint3(pb, g, st, 2)
    return pb, g, st, adj


@pytest.mark.parametrize("path", ["auto", "step"])
def test_config4_full_size_short_marches(path, config4_oracle_short):
    """192^3, FP32, on the warp-column kernels (auto) and the plane-march kernels
    (step): three forward steps from rest and two adjoint iterations on that state
    against the oracle's, over the whole lattice (relative L2) and at sampled faces,
    box edges, corners and interior nodes (max error of a node against the field's
    scale)."""
    pb, g, st, adj = config4_oracle_short
    s = LKS(pb, real="f32", path=path)
    s.lks_forward(torch.from_numpy(g))
    s.alks_adjoint()
    q = s.query()
    assert q.fwd_path == (3 if path == "auto" else 1) and q.adj_path == q.fwd_path and q.device_status == 0
    cur = [f.double().cpu().numpy() for f in s.get_state()]
    ref = [st.rho - 1.0, st.u, st.v, st.w]
    for c in range(4):
        assert rel_l2(cur[c], ref[c]) <= 1e-5, c
    a = np.stack([x.double().cpu().numpy() for x in s.get_adjoint()])
    for k in range(O.NADJ3):
        assert rel_l2(a[k], adj[k]) <= 1e-5, O.ADJ3_NAMES[k]
    nodes = _sample_nodes(pb, np.random.default_rng(4))
    scale = max(np.abs(ref[1]).max(), 1e-30)
    ascale = np.abs(adj).reshape(O.NADJ3, -1).max(axis=1) + 1e-30
    for (i, j, kz) in nodes:
        assert abs(cur[0][kz, j, i] - ref[0][kz, j, i]) <= 2e-6, (i, j, kz)
        for c in range(1, 4):
            assert abs(cur[c][kz, j, i] - ref[c][kz, j, i]) <= 2e-5 * scale, (i, j, kz, c)
        for k in range(O.NADJ3):
            assert abs(a[k, kz, j, i] - adj[k, kz, j, i]) <= 2e-5 * ascale[k], (i, j, kz, O.ADJ3_NAMES[k])
