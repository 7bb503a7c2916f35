"""GPU parity of the batched form (lks_batch_*): many unsteady designs of unequal
size in one persistent launch per step, the whole gradient one CUDA graph launch.

Each design's gradient is compared with the FP64 oracle (Steps 2-5 of Sec. 2.7
for an unsteady problem), with the single-lattice library path on the same
inputs (bit for bit where that path runs the same TMA kernels), across the tile
shapes the autotuner chooses from, and between the graph and direct launches.
The designs cover ragged tiles, nx not a multiple of four, a lattice smaller than
every tile shape, a ragged last checkpoint segment and a single segment.
"""
import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_2411_03090_gb300 import LKS, LKSBatch  # noqa: E402


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def designs(n_steps=60):
    kw = dict(steady=False, n_steps=n_steps, n_adj=n_steps, pulse_mean=0.75, pulse_amp=0.25, pulse_period=40.0,
              sigma=2.0, strip=2)
    return [
        inputs.channel(136, 40, Re=10.0, seed=31, **kw),  # nx % 4 == 0: the single path runs TMA kernels
        inputs.channel(70, 33, Re=25.0, seed=32, **kw),   # nx % 4 != 0, ragged tiles both ways
        inputs.channel(20, 12, Re=5.0, seed=33, **kw),    # smaller than every tile shape
        inputs.channel(200, 24, Re=40.0, seed=34, **kw),  # wide and flat
    ]


def gammas(pbs):
    return [torch.from_numpy(p.gamma()).float().cuda() for p in pbs]


def run(pbs, **kw):
    b = LKSBatch(pbs, **kw)
    J, grads = b.gradient(gammas(pbs))
    torch.cuda.synchronize()
    st = b.query()
    assert st.device_status == 0
    return J.cpu().numpy().copy(), [g.double().cpu().numpy().copy() for g in grads], st


@pytest.fixture(scope="module")
def oracle_refs():
    pbs = designs()
    return pbs, [O.unsteady_gradient(p, p.gamma()) for p in pbs]


def test_batch_matches_oracle(oracle_refs):
    pbs, refs = oracle_refs
    J, grads, st = run(pbs, checkpoint_every=7, snapshot="f32", tile_config=0)
    assert st.n_ckpt == 9 and st.checkpoint_every == 7  # 60 = 8 x 7 + 4: ragged last segment
    for k, ref in enumerate(refs):
        assert abs(J[k] - ref["J"]) <= 1e-5 * abs(ref["J"]), k
        assert rel_l2(grads[k], ref["dJdgamma"]) <= 1e-3, k


def test_batch_bf16_snapshots_match_oracle(oracle_refs):
    """Reduced-precision checkpoints (per design and field max-abs scale) keep the
    gradient within the FP32 tolerance of the FP64 oracle."""
    pbs, refs = oracle_refs
    for snap in ("bf16", "f16"):
        J, grads, _ = run(pbs, checkpoint_every=7, snapshot=snap, tile_config=0)
        for k, ref in enumerate(refs):
            assert abs(J[k] - ref["J"]) <= 1e-5 * abs(ref["J"]), (snap, k)
            assert rel_l2(grads[k], ref["dJdgamma"]) <= 1e-3, (snap, k)


def test_batch_equals_single_lattice_path():
    """Same per-node arithmetic as the single-lattice TMA kernels: identical
    gradients; J differs only in the order of its FP64 partial sums."""
    pbs = designs()
    J, grads, _ = run(pbs, checkpoint_every=7, snapshot="f32", tile_config=0)
    pb = pbs[0]
    s = LKS(pb, real="f32", checkpoint_every=7, snapshot="f32")
    Js, gs = s.gradient(torch.from_numpy(pb.gamma()).float().cuda())
    assert s.query().fwd_path == 1
    np.testing.assert_array_equal(grads[0], gs.double().cpu().numpy())
    assert abs(J[0] - Js.item()) <= 1e-12 * abs(Js.item())


def test_batch_tile_shapes_agree():
    """Every tile shape computes each node the same way: identical gradients."""
    pbs = designs()
    J0, g0, _ = run(pbs, checkpoint_every=7, snapshot="bf16", tile_config=0)
    for c in (1, 2, 3):
        J, g, st = run(pbs, checkpoint_every=7, snapshot="bf16", tile_config=c)
        assert st.tile_config == c
        for k in range(len(pbs)):
            np.testing.assert_array_equal(g[k], g0[k])
            assert abs(J[k] - J0[k]) <= 1e-12 * abs(J0[k])


def test_batch_column_kernels_equal_tma_kernels():
    """The warp-column forward (60 x 40 tiles, two columns per lane) and adjoint
    (28 x 32 tiles) compute each node with the arithmetic of the TMA-staged kernels,
    also for an odd nx (the forward's last lane pair half outside its design):
    identical gradients; J differs only in the order of its FP64 partial sums.  The
    odd designs also match the oracle."""
    kw = dict(steady=False, n_steps=60, n_adj=60, pulse_mean=0.75, pulse_amp=0.25, pulse_period=40.0,
              sigma=2.0, strip=2)
    pbs = designs() + [inputs.channel(45, 30, Re=15.0, seed=35, **kw), inputs.channel(131, 85, Re=30.0, seed=36, **kw)]
    Jt, gt, st = run(pbs, checkpoint_every=7, snapshot="f32", tile_config=0, fwd_column=0, adj_column=0)
    Jc, gc, sc = run(pbs, checkpoint_every=7, snapshot="f32", tile_config=0, fwd_column=1, adj_column=1)
    assert st.fwd_column == 0 and sc.fwd_column == 1 and st.adj_column == 0 and sc.adj_column == 1
    for k in range(len(pbs)):
        np.testing.assert_array_equal(gc[k], gt[k])
        assert abs(Jc[k] - Jt[k]) <= 1e-12 * abs(Jt[k]), k
    for k in (4, 5):
        ref = O.unsteady_gradient(pbs[k], pbs[k].gamma())
        assert abs(Jc[k] - ref["J"]) <= 1e-5 * abs(ref["J"]), k
        assert rel_l2(gc[k], ref["dJdgamma"]) <= 1e-3, k


def test_batch_graph_equals_direct_launches():
    pbs = designs()
    Jg, gg, sg = run(pbs, checkpoint_every=13, snapshot="bf16", tile_config=1, use_graph=True)
    Jd, gd, sd = run(pbs, checkpoint_every=13, snapshot="bf16", tile_config=1, use_graph=False)
    assert sg.graph == 1 and sd.graph == 0
    assert sg.kernel_launches == sd.kernel_launches > 0
    np.testing.assert_array_equal(Jg, Jd)
    for a, b in zip(gg, gd):
        np.testing.assert_array_equal(a, b)


def test_batch_single_segment_and_autotune():
    """K >= n_steps (one segment), the autotuned tile shape, and one design."""
    pbs = designs(n_steps=25)[1:2]
    ref = O.unsteady_gradient(pbs[0], pbs[0].gamma())
    J, grads, st = run(pbs, checkpoint_every=100, snapshot="f32")
    assert st.n_ckpt == 1 and st.checkpoint_every == 25
    assert all(t > 0 for t in st.tune_us) and st.tune_col_us > 0 and st.tune_acol_us > 0
    # per level: two forward steps and one adjoint step, each on its faster kernel
    fwd, lvl = np.array(list(st.tune_fwd_us)), np.array(list(st.tune_us))
    adj = lvl - 2 * fwd
    cost = 2 * np.minimum(fwd, st.tune_col_us) + np.minimum(adj, st.tune_acol_us)
    assert st.tile_config == int(np.argmin(cost))
    assert st.fwd_column == int(st.tune_col_us < fwd[st.tile_config])
    assert st.adj_column == int(st.tune_acol_us < adj[st.tile_config])
    assert abs(J[0] - ref["J"]) <= 1e-5 * abs(ref["J"])
    assert rel_l2(grads[0], ref["dJdgamma"]) <= 1e-3


def test_batch_repeated_calls_take_new_inputs():
    """The graph replays with the pointers of each call: a second call with other
    designs' fields gives what a fresh handle gives for them."""
    pbs = designs()
    b = LKSBatch(pbs, checkpoint_every=9, snapshot="bf16", tile_config=2)
    g1 = gammas(pbs)
    J1, gr1 = b.gradient(g1)
    J1 = J1.cpu().numpy().copy()
    gr1 = [g.cpu().numpy().copy() for g in gr1]
    g2 = [torch.clamp(g * 0.7 + 0.2, 0.0, 1.0) for g in g1]
    J2, gr2 = b.gradient(g2)
    J2 = J2.cpu().numpy().copy()
    gr2 = [g.cpu().numpy().copy() for g in gr2]
    fresh = LKSBatch(pbs, checkpoint_every=9, snapshot="bf16", tile_config=2)
    J3, gr3 = fresh.gradient(g2)
    np.testing.assert_array_equal(J2, J3.cpu().numpy())
    for a, c in zip(gr2, gr3):
        np.testing.assert_array_equal(a, c.cpu().numpy())
    J4, gr4 = b.gradient(g1)
    np.testing.assert_array_equal(J1, J4.cpu().numpy())
    assert not np.array_equal(J1, J2)
    assert b.query().gradients == 3


def test_batch_config5_full_size_sampled():
    """The 64-design batch at full size (5000 steps, BF16 snapshots, autotuned tile
    shape, graph launch), as the benchmark times it; the two smallest designs are
    recomputed by the FP64 oracle and compared."""
    pbs = inputs.config5()
    b = LKSBatch(pbs, snapshot="bf16")
    J, grads = b.gradient(gammas(pbs))
    torch.cuda.synchronize()
    st = b.query()
    assert st.device_status == 0 and st.graph == 1
    J = J.cpu().numpy()
    assert np.all(np.isfinite(J)) and np.all(J > 0)
    order = np.argsort([p.nx * p.ny for p in pbs])[:2]
    for k in order:
        ref = O.unsteady_gradient(pbs[k], pbs[k].gamma())
        assert abs(J[k] - ref["J"]) <= 1e-4 * abs(ref["J"]), k
        assert rel_l2(grads[k].double().cpu().numpy(), ref["dJdgamma"]) <= 1e-3, k
