"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
entry point that include/lks.h declares, validates descriptors, and its
generalized-inverse edge maps equal the paper's closed form and the oracle."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import inputs
from oracle import oracle as O
from paper_2411_03090_gb300 import lks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _declared():
    src = open(os.path.join(ROOT, "include", "lks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:lks|alks)_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = lks.load()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(lks.EXPORTS)


def test_status_strings():
    L = lks.load()
    for s in range(8):
        assert L.lks_status_string(s)


def _moments(f):
    return np.array([W @ f, W @ (CX * f), W @ (CY * f), W @ (CX * CX * f), W @ (CX * CY * f),
                     W @ (CY * CY * f)])


@pytest.mark.parametrize("A", [-0.6675, 0.17625, 0.3])
def test_bottom_face_map_is_eq_ftilde(A):
    """Moments of the bottom-face fill equal those of Eq. (ftilde) (Sec. 2.5)."""
    M = lks.edge_moment_map(A, 3)[:, :9]
    rng = np.random.default_rng(0)
    f = rng.standard_normal(9)
    f[[4, 7, 8]] = 0.0
    full = f.copy()
    full[4] = (f[2] + f[5] + f[6]) / 3
    full[7] = (4 * f[2] + 7 * f[5] + f[6]) / 12
    full[8] = (4 * f[2] + f[5] + 7 * f[6]) / 12
    np.testing.assert_allclose(M @ f, _moments(full), atol=1e-14)


@pytest.mark.parametrize("cls,n,pressure", [(0, (-1, 0), 0), (1, (1, 0), 1), (2, (1, 0), 0),
                                            (3, (0, -1), 0), (4, (0, 1), 0), (5, (-1, -1), 0),
                                            (6, (1, -1), 0), (7, (-1, 1), 0), (8, (1, 1), 0)])
def test_edge_maps_match_oracle(cls, n, pressure):
    A = -0.2
    M = lks.edge_moment_map(A, cls)
    rng = np.random.default_rng(cls)
    unknown = np.array([1 if (CX[k] * n[0] > 0 or CY[k] * n[1] > 0) else 0 for k in range(9)])
    f = rng.standard_normal(9) * (1 - unknown)
    kT = 0.37
    full, _ = O.bc_flow(n, pressure, A, f, unknown, kT=kT)
    np.testing.assert_allclose(M[:, :9] @ f + M[:, 9] * kT, _moments(full), atol=1e-13)
    # a boundary objective term in every residual row (the static pressure drop)
    jb = -0.61
    Mj = lks.edge_objective_map(A, cls)
    full_j, _ = O.bc_flow(n, pressure, A, f, unknown, kT=kT, jb=jb)
    np.testing.assert_allclose(M[:, :9] @ f + M[:, 9] * kT + Mj * jb, _moments(full_j), atol=1e-13)


def test_descriptor_validation():
    pb = inputs.config1()
    d = lks.make_desc(pb)
    assert lks.workspace_size(d) > 0
    for field, val in (("nx", 3), ("real_type", 7), ("nu", 0.9), ("version", 99), ("version", 1), ("n_steps", 0),
                       ("res_steps", 4), ("res_steps", -1), ("warm_start", 2), ("segment_type", 7),
                       ("segment_type", 1)):  # a 16-bit segment needs an unsteady problem
        bad = lks.make_desc(pb)
        setattr(bad, field, val)
        with pytest.raises(lks.LKSError) as e:
            lks.workspace_size(bad)
        assert e.value.status == 1
    for q in range(4):
        bad = lks.make_desc(pb)
        bad.reserved[q] = 1
        with pytest.raises(lks.LKSError):
            lks.workspace_size(bad)
    bad = lks.make_desc(pb.with_(steady=False))
    bad.warm_start = 1  # warm starts are for steady marches
    with pytest.raises(lks.LKSError):
        lks.workspace_size(bad)
    assert lks.workspace_size(lks.make_desc(pb, warm_start=True)) == lks.workspace_size(d)
    ok = lks.make_desc(pb.with_(kappa_p=1.0))  # steady D2Q9: the pressure drop is accepted
    assert ok.kappa_p == 1.0 and lks.workspace_size(ok) == lks.workspace_size(d)
    bad = lks.make_desc(pb.with_(kappa_p=1.0, steady=False))  # unsteady D2Q9: not with kappa_p
    with pytest.raises(lks.LKSError):
        lks.workspace_size(bad)
    # the energy loss: D2Q9, steady or unsteady, on the per-step kernels
    for st in (True, False):
        ok = lks.make_desc(pb.with_(kappa_E=1.0, steady=st))
        assert ok.kappa_E == 1.0 and lks.workspace_size(ok) > 0
    for path in ("column", "resident"):
        with pytest.raises(lks.LKSError):
            lks.workspace_size(lks.make_desc(pb.with_(kappa_E=1.0), path=path))
    bad = lks.make_desc(pb.with_(kappa_E=1.0))
    bad.kappa_E = float("inf")
    with pytest.raises(lks.LKSError):
        lks.workspace_size(bad)
    d3 = lks.make_desc(inputs.config4())
    d3.kappa_E = 1.0  # D3Q19: not built
    with pytest.raises(lks.LKSError):
        lks.workspace_size(d3)
    d3 = lks.make_desc(inputs.config4())
    assert d3.kappa_p == 1.0 and lks.workspace_size(d3) > 0
    d3.kappa_p = float("nan")
    with pytest.raises(lks.LKSError):
        lks.workspace_size(d3)
    d3 = lks.make_desc(inputs.config4(), tol=1e-6, max_steps=5000)  # D3Q19: fixed counts only
    with pytest.raises(lks.LKSError):
        lks.workspace_size(d3)
    assert lks.workspace_size(lks.make_desc(pb, tol=1e-6, max_steps=pb.n_steps)) > 0
    for kw in (dict(tol=-1.0), dict(tol=1e-6, max_steps=pb.n_steps - 1), dict(tol=float("inf"), max_steps=10**6)):
        with pytest.raises(lks.LKSError):
            lks.workspace_size(lks.make_desc(pb, **kw))
    unsteady = inputs.config3().with_(nx=64, ny=32, n_steps=100)
    with pytest.raises(lks.LKSError):
        lks.workspace_size(lks.make_desc(unsteady, tol=1e-6, max_steps=1000))
    for ks in (1, 2, 3):
        assert lks.workspace_size(lks.make_desc(pb, res_steps=ks)) == lks.workspace_size(d)


@pytest.mark.parametrize("field,val", [("nx", 0), ("ny", 0), ("nx", -8), ("ny", 4), ("nz", 2), ("n_adj", 0),
                                       ("checkpoint_every", -1), ("snapshot_type", 3), ("exec_path", 4),
                                       ("exec_path", -1), ("nu", float("nan")), ("nu", 0.5), ("q_alpha", 0.0),
                                       ("in_y0", -1), ("in_y1", 10**6), ("out_y0", 0)])
def test_degenerate_descriptors_are_refused(field, val):
    """Empty, negative and out-of-range fields of a D2Q9 descriptor: refused with
    LKS_ERR_INVALID_ARG before any device work."""
    bad = lks.make_desc(inputs.config1())
    setattr(bad, field, val)
    n = C.c_size_t(123)
    assert lks.load().lks_workspace_size(C.byref(bad), C.byref(n)) == 1


@pytest.mark.parametrize("field,val", [("nx", 4), ("nz", 0), ("nz", -3), ("n_steps", 0), ("n_adj", 0),
                                       ("res_steps", 1), ("warm_start", 1), ("thermal", 1)])
def test_degenerate_d3q19_descriptors_are_refused(field, val):
    bad = lks.make_desc(inputs.config4())
    setattr(bad, field, val)
    with pytest.raises(lks.LKSError) as e:
        lks.workspace_size(bad)
    assert e.value.status == 1


def test_largest_lattices_are_sized_without_overflow():
    """The node count is limited to 2^31 (the kernels' node indices); at that limit the
    workspace is computed in 64-bit arithmetic: it grows with the lattice and holds at
    least two levels of the state and of the adjoint fields of every node."""
    pb = inputs.config1()
    small = lks.make_desc(pb)
    big = lks.make_desc(pb)
    big.nx, big.ny = 46340, 46340  # 2.147e9 nodes, just under 2^31
    big.in_y0, big.in_y1, big.out_y0, big.out_y1 = 0, 46339, 1, 46338
    n_small, n_big = lks.workspace_size(small), lks.workspace_size(big)
    nodes = 46340 * 46340
    assert n_big > n_small and n_big >= nodes * 4 * 2 * (3 + 6)  # FP32: delta-rho, u, v and six adjoint fields
    over = lks.make_desc(pb)
    over.nx, over.ny = 65536, 32769  # 2^31 + 65536 nodes
    over.in_y0, over.in_y1, over.out_y0, over.out_y1 = 0, 32768, 1, 32767
    with pytest.raises(lks.LKSError):
        lks.workspace_size(over)
    d3 = lks.make_desc(inputs.config4())
    d3.nx = d3.ny = d3.nz = 1291  # 2.15e9 nodes > 2^31
    with pytest.raises(lks.LKSError):
        lks.workspace_size(d3)
    d3.nx = d3.ny = d3.nz = 1290  # 2.147e9 nodes
    # FP32: two levels of delta-rho, u, v, w and of the ten adjoint fields, and four coefficient fields
    assert lks.workspace_size(d3) >= 1290 ** 3 * 4 * (2 * (4 + 10) + 4)


def test_workspace_grows_with_checkpoint_storage():
    p3 = inputs.config3().with_(nx=64, ny=32, n_steps=1000)
    plain = lks.workspace_size(lks.make_desc(p3, checkpoint_every=0))
    ck = lks.workspace_size(lks.make_desc(p3, checkpoint_every=100, snapshot="bf16"))
    assert ck < plain


def test_selftest_wait_rejects_bad_arguments_without_gpu_work():
    L = lks.load()
    rec = C.c_int32(-1)
    assert L.lks_selftest_wait(2, C.c_void_p(16), None, C.byref(rec)) == 1
    assert L.lks_selftest_wait(0, None, None, C.byref(rec)) == 1
    assert L.lks_selftest_wait(1, C.c_void_p(16), None, None) == 1
    assert rec.value == -1


def test_noalloc_rejects_tolerance_marches_without_gpu_work():
    """lks_gradient_noalloc never synchronises, so a descriptor asking for a
    tolerance march (which reads its change back) is refused before any GPU work."""
    L = lks.load()
    pb = inputs.config1()
    d = lks.make_desc(pb, tol=1e-6, max_steps=pb.n_steps)
    p = C.c_void_p(256)
    assert L.lks_gradient_noalloc(C.byref(d), p, C.cast(p, C.POINTER(C.c_double)), p, None) == 1


def test_create_rejects_bad_workspace_without_gpu_work():
    L = lks.load()
    d = lks.make_desc(inputs.config1())
    h = C.c_void_p()
    st = L.lks_create(C.byref(d), None, C.c_size_t(16), None, C.byref(h))
    assert st == 2 and not h.value


def _cuda_device_present():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


@pytest.mark.skipif(_cuda_device_present(), reason="drives the error paths a machine without a GPU takes")
@pytest.mark.parametrize("kw", [dict(), dict(steady=False, pulse_mean=0.75, pulse_amp=0.25, pulse_period=10.0),
                                dict(steady=False, pulse_mean=0.75, pulse_amp=0.25, pulse_period=10.0,
                                     checkpoint_every=5)])
def test_create_without_a_gpu_fails_with_cuda_error_and_message(kw):
    """Without a GPU every CUDA call fails: lks_create (steady, plain unsteady, and
    checkpointed unsteady, which also creates its own stream and events) must return
    LKS_ERR_CUDA, hand back no handle and not crash.  The workspace is a correctly
    sized, aligned host buffer that the library never reaches."""
    L = lks.load()
    ck = kw.pop("checkpoint_every", 0)
    pb = inputs.channel(24, 12, Re=10.0, seed=1, n_steps=20, n_adj=20, **kw)
    d = lks.make_desc(pb, checkpoint_every=ck, snapshot="bf16") if ck else lks.make_desc(pb)
    n = C.c_size_t(0)
    assert L.lks_workspace_size(C.byref(d), C.byref(n)) == 0 and n.value > 0
    raw = np.zeros(n.value + 256, dtype=np.uint8)
    base = raw.ctypes.data
    ws = C.c_void_p(base + (-base) % 256)
    h = C.c_void_p()
    st = L.lks_create(C.byref(d), ws, C.c_size_t(n.value), None, C.byref(h))
    assert st == 3 and not h.value  # LKS_ERR_CUDA


# ---------------------------------------------------------------------------------------
# Batched form: host-side planning (no GPU work)
# ---------------------------------------------------------------------------------------
def _batch(n_steps=120):
    kw = dict(steady=False, n_steps=n_steps, n_adj=n_steps, pulse_mean=0.75, pulse_amp=0.25, pulse_period=50.0)
    return [inputs.channel(130, 70, Re=50.0, seed=10, **kw), inputs.channel(256, 64, Re=20.0, seed=11, **kw),
            inputs.channel(33, 20, Re=10.0, seed=12, **kw)]


def _bsize(descs, opt):
    n = C.c_size_t(0)
    st = lks.load().lks_batch_workspace_size(len(descs), descs, C.byref(opt) if opt is not None else None,
                                             C.byref(n))
    return st, n.value


def test_batch_workspace_validation():
    pbs = _batch()
    ok = lks.batch_descs(pbs)
    st, n = _bsize(ok, None)
    assert st == 0 and n > 0
    for mutate in (lambda d: setattr(d[1], "steady", 1), lambda d: setattr(d[0], "thermal", 1),
                   lambda d: setattr(d[2], "real_type", 1), lambda d: setattr(d[1], "n_steps", 119),
                   lambda d: setattr(d[0], "nu", 0.9)):
        d = lks.batch_descs(pbs)
        mutate(d)
        assert _bsize(d, None)[0] == 1
    for field, val in (("version", 7), ("tile_config", 4), ("snapshot_type", 3), ("use_graph", 2),
                       ("checkpoint_every", -1), ("fwd_column", 2), ("fwd_column", -2), ("adj_column", 2)):
        o = lks.batch_options()
        setattr(o, field, val)
        assert _bsize(ok, o)[0] == 1, field
    o = lks.batch_options()
    o.reserved[2] = 1
    assert _bsize(ok, o)[0] == 1
    assert lks.load().lks_batch_workspace_size(0, ok, None, C.byref(C.c_size_t())) == 1


def test_batch_memory_optimal_checkpoint_spacing():
    """K = 0 picks the spacing with the least workspace; the snapshot width and the
    number of designs enter as expected."""
    pbs = _batch()
    d = lks.batch_descs(pbs)
    auto = _bsize(d, lks.batch_options(checkpoint_every=0))[1]
    for K in (1, 2, 5, 9, 10, 11, 12, 20, 60, 120, 500):
        assert auto <= _bsize(d, lks.batch_options(checkpoint_every=K))[1], K
    bf = _bsize(d, lks.batch_options(checkpoint_every=10, snapshot="bf16"))[1]
    f32 = _bsize(d, lks.batch_options(checkpoint_every=10, snapshot="f32"))[1]
    assert bf < f32
    assert _bsize(lks.batch_descs(pbs[:2]), None)[1] < auto


def test_batch_create_rejects_bad_workspace_without_gpu_work():
    L = lks.load()
    d = lks.batch_descs(_batch())
    h = C.c_void_p()
    assert L.lks_batch_create(3, d, None, None, C.c_size_t(16), None, C.byref(h)) == 2 and not h.value
    o = lks.batch_options()
    o.tile_config = 9
    assert L.lks_batch_create(3, d, C.byref(o), None, C.c_size_t(16), None, C.byref(h)) == 1 and not h.value


def test_config5_recipe():
    pbs = inputs.config5()
    assert len(pbs) == 64
    assert all(128 <= p.nx <= 512 and 64 <= p.ny <= 256 for p in pbs)
    assert all(0.012 <= p.nu <= 0.30 for p in pbs)
    Re = [p.u_max * (p.ny - 1) / p.nu for p in pbs]
    assert all(20.0 - 1e-9 <= r <= 200.0 + 1e-9 for r in Re)
    assert [p.seed for p in pbs] == list(range(500, 564))
    assert all(p.n_steps == 5000 and not p.steady for p in pbs)
