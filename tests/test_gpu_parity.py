"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: the FP64 instance of the kernels agrees with the oracle to rounding
(<= 1e-10 relative); the FP32 path keeps fields within 1e-5 relative L2 and
gradients within 1e-3 relative L2 of the oracle.
"""
import numpy as np
import pytest
import torch

import inputs
from oracle import oracle as O

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2411_03090_gb300 import LKS, LKSError  # noqa: E402
from paper_2411_03090_gb300.autograd import objective  # noqa: E402


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def small(steady=True, nx=70, **kw):
    """70 x 40 nodes: three tiles across x and y with ragged last tiles (plain
    per-step kernels).  nx = 136: a multiple of four, so the FP32 per-step marches
    run the TMA-staged kernels, again with ragged last tiles (136 = 2 x 64 + 8)."""
    base = dict(seed=1, sigma=2.0, strip=2, n_steps=300, n_adj=300)
    base.update(kw)
    if not steady:
        base.update(steady=False, pulse_mean=0.75, pulse_amp=0.25, pulse_period=120.0)
    return inputs.channel(nx, 40, Re=10.0, **base)


def oracle_state(st):
    return [st.rho - 1.0, st.u, st.v]


def f32(a):
    """An array rounded to FP32 and back: the oracle and the FP32 kernels then start
    a step from exactly the same values."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def oracle_developed_state(pb, g, n):
    """The oracle's state after n steps from rest, rounded to FP32 (drho rounded as
    stored, rho - 1)."""
    st, _, _, _ = O.forward(pb, g, n)
    r = O.State(pb.ny, pb.nx)
    r.rho, r.u, r.v, r.T = 1.0 + f32(st.rho - 1.0), f32(st.u), f32(st.v), f32(st.T)
    return r


def set_gpu_state(s, g, st, t):
    z = lambda a: torch.from_numpy(np.ascontiguousarray(a))  # noqa: E731
    s.set_state(z(g), z(st.rho - 1.0), z(st.u), z(st.v), z(st.T), t=t)


def gpu_state(s):
    d, u, v, T = [x.double().cpu().numpy() for x in s.get_state()]
    return [d, u, v], T


# ---------------------------------------------------------------------------------------
# Forward
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("path", ["step", "resident"])
@pytest.mark.parametrize("real,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_forward_matches_oracle(real, tol, path):
    pb = small()
    g = pb.gamma()
    s = LKS(pb, real=real, path=path)
    J = s.lks_forward(torch.from_numpy(g)).item()
    st, _, _, _ = O.forward(pb, g, pb.n_steps)
    got, _ = gpu_state(s)
    for a, b in zip(got, oracle_state(st)):
        assert rel_l2(a, b) <= tol
    assert abs(J - O.objective(pb, g, st)) <= tol * abs(J)


def test_tolerance_march_matches_oracle_at_the_same_step_count():
    """tol > 0: chunks of n_steps with one measured step after each until the
    relative change of a step is <= tol.  The state equals the oracle's after the
    number of steps the library reports, the reported change is the oracle's
    max |du| + |dv| of that step over max |u| + |v|, and the adjoint likewise."""
    pb = small(n_steps=200, n_adj=200)
    g = pb.gamma()
    s = LKS(pb, real="f64", path="step", tol=1e-7, max_steps=60000)
    s.lks_forward(torch.from_numpy(g))
    q = s.query()
    n = q.forward_steps
    assert n % 201 == 0 and 0 < q.fwd_change <= 1e-7
    st_prev, _, _, _ = O.forward(pb, g, n - 1)
    st, _, _, _ = O.forward(pb, g, 1, state=st_prev)
    got, _ = gpu_state(s)
    for a, b in zip(got, oracle_state(st)):
        assert rel_l2(a, b) <= 1e-11
    change = (np.abs(st.u - st_prev.u) + np.abs(st.v - st_prev.v)).max() / (np.abs(st.u) + np.abs(st.v)).max()
    assert abs(q.fwd_change - change) <= 1e-6 * change  # the library takes the maxima in FP32
    s.alks_adjoint()
    q = s.query()
    m = q.adjoint_steps
    assert m % 201 == 0 and 0 < q.adj_change <= 1e-7
    adj, _, _ = O.steady_adjoint(pb, g, st, m)
    got_a = [a.double().cpu().numpy() for a in s.get_adjoint()]
    for qq in range(6):
        assert rel_l2(got_a[qq], adj[qq]) <= 1e-10, qq


def test_tolerance_march_on_the_resident_path():
    """FP32, steady: the chunks run on the resident march and each measured step on
    the per-step kernels; the state after the reported number of steps equals the
    oracle's to FP32 tolerance."""
    pb = inputs.channel(128, 64, Re=10.0, seed=2, sigma=2.0, strip=2, n_steps=500, n_adj=500)
    g = pb.gamma()
    s = LKS(pb, real="f32", path="auto", tol=1e-4, max_steps=40000)
    s.lks_forward(torch.from_numpy(g))
    q = s.query()
    assert q.fwd_path == 2 and q.forward_steps % 501 == 0 and q.fwd_change <= 1e-4
    st, _, _, _ = O.forward(pb, g, q.forward_steps)
    got, _ = gpu_state(s)
    for a, b in zip(got[1:], oracle_state(st)[1:]):
        assert rel_l2(a, b) <= 1e-5


def test_tolerance_not_reached_reports_not_converged():
    """A tolerance the march cannot reach within max_steps: LKS_ERR_NOT_CONVERGED after
    exactly max_steps steps (chunks 100 + 1 + 100 + 1 + 47 + 1), state and J in place."""
    pb = small(n_steps=100, n_adj=100)
    g = torch.from_numpy(pb.gamma())
    s = LKS(pb, real="f64", path="step", tol=1e-30, max_steps=250)
    with pytest.raises(LKSError) as e:
        s.lks_forward(g)
    assert e.value.status == 5
    q = s.query()
    assert q.forward_steps == 250 and q.fwd_change > 0 and q.device_status == 0
    st, _, _, _ = O.forward(pb, pb.gamma(), 250)
    got, _ = gpu_state(s)
    for a, b in zip(got, oracle_state(st)):
        assert rel_l2(a, b) <= 1e-12


@pytest.mark.parametrize("nu", [0.1, 0.315])
def test_poiseuille_on_gpu(nu):
    """Empty channel converges to the exact Poiseuille profile (FP64 instance)."""
    pb = inputs.poiseuille(70, 33, nu=nu, u_max=0.02).with_(n_steps=30000)
    s = LKS(pb, real="f64")
    s.lks_forward(torch.ones(pb.ny, pb.nx, dtype=torch.float64))
    (d, u, v), _ = gpu_state(s)
    H = pb.ny - 1
    y = np.arange(pb.ny)
    U = 4 * pb.u_max * y * (H - y) / H ** 2
    assert np.abs(u - U[:, None]).max() <= 1e-9 * pb.u_max
    assert np.abs(v).max() <= 1e-9 * pb.u_max


def test_single_step_full_size_config2():
    """512 x 256 (the benchmark lattice), FP32, launch configuration of the bench:
    one step from a developed state (the oracle's, after 400 steps, rounded to FP32)
    equals the oracle's step from the same state."""
    pb = inputs.config2()
    g = pb.gamma()
    st = oracle_developed_state(pb, g, 400)
    s = LKS(pb, real="f32")
    set_gpu_state(s, g, st, 400)
    d0 = st.rho - 1.0
    s.march(1)
    (d1, u1, v1), _ = gpu_state(s)
    ref = O.forward_step(pb, f32(g), 401, st)
    for a, b, scale in ((d1, ref.rho - 1.0, np.abs(d0).max()), (u1, ref.u, pb.u_max),
                        (v1, ref.v, pb.u_max)):
        assert np.abs(a - b).max() <= 2e-6 * scale


# ---------------------------------------------------------------------------------------
# Adjoint and sensitivity
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("path", ["step", "resident"])
@pytest.mark.parametrize("real,ftol,gtol", [("f64", 1e-11, 1e-10), ("f32", 1e-5, 1e-3)])
def test_steady_gradient_matches_oracle(real, ftol, gtol, path):
    pb = small()
    g = pb.gamma()
    s = LKS(pb, real=real, path=path)
    J, grad = s.gradient(torch.from_numpy(g))
    ref = O.steady_gradient(pb, g)
    assert abs(J.item() - ref["J"]) <= ftol * abs(ref["J"])
    adj = [a.double().cpu().numpy() for a in s.get_adjoint()[:6]]
    for q in range(6):
        assert rel_l2(adj[q], ref["adjoint"][q]) <= gtol, q
    assert rel_l2(grad.double().cpu().numpy(), ref["dJdgamma"]) <= gtol
    assert s.query().device_status == 0


@pytest.mark.parametrize("real,ftol,jtol,gtol", [("f64", 1e-11, 1e-11, 1e-10),
                                                 ("f32", 1e-5, 1e-5, 1e-3)])
def test_config1_full(real, ftol, jtol, gtol):
    """64 x 64, Re = 10 (nu = 0.315, A < 0), 5000 forward + 5000 adjoint steps.
    Fields within ftol relative L2, J within jtol relative, gradient within gtol
    (measured in FP32: fields 2e-6, J 3.4e-6, gradient 3.3e-6)."""
    pb = inputs.config1()
    g = pb.gamma()
    s = LKS(pb, real=real)
    J, grad = s.gradient(torch.from_numpy(g))
    ref = O.steady_gradient(pb, g)
    got, _ = gpu_state(s)
    for a, b in zip(got, oracle_state(ref["state"])):
        assert rel_l2(a, b) <= ftol
    assert abs(J.item() - ref["J"]) <= jtol * abs(ref["J"])
    assert rel_l2(grad.double().cpu().numpy(), ref["dJdgamma"]) <= gtol


def test_single_adjoint_step_full_size_config2():
    """512 x 256, FP32: one ALKS step from developed adjoint fields (the oracle's
    state after 300 steps and adjoint after 200 iterations, rounded to FP32) equals
    the oracle's step from the same fields."""
    pb = inputs.config2()
    g = pb.gamma()
    gf = f32(g)
    st = oracle_developed_state(pb, g, 300)
    adj, _, _ = O.steady_adjoint(pb, gf, st, 200)
    full = np.zeros((9, pb.ny, pb.nx))
    full[:6] = f32(adj[:6])
    s = LKS(pb, real="f32")
    set_gpu_state(s, g, st, 300)
    s.set_adjoint([torch.from_numpy(np.ascontiguousarray(full[q])) for q in range(6)])
    s.adjoint_march(1)
    a1 = [a.double().cpu().numpy() for a in s.get_adjoint()[:6]]
    ref = O.adjoint_step(pb, gf, st, st, full)
    for q in range(6):
        scale = np.abs(ref[q]).max()
        assert np.abs(a1[q] - ref[q]).max() <= 1e-5 * scale, q


def test_bench_path_full_size_config2_matches_oracle():
    """The benchmark's launch configuration at full size: 512 x 256 on the resident
    marches (64 x 14 tiles, one per SM), 2000 forward + 2000 adjoint steps, against
    the FP64 oracle element by element: state fields within 1e-5 relative L2 (the
    field tolerance), the six adjoint fields and dJ/dgamma within 1e-3 (the gradient
    tolerance; measured 2e-6 for the state, 8e-6 for the adjoint, 3e-6 for the
    gradient)."""
    pb = inputs.config2().with_(n_steps=2000, n_adj=2000)
    g = pb.gamma()
    s = LKS(pb, real="f32", path="auto")
    J, grad = s.gradient(torch.from_numpy(g))
    q = s.query()
    assert q.fwd_path == 2 and q.adj_path == 2 and q.device_status == 0
    ref = O.steady_gradient(pb, g)
    got, _ = gpu_state(s)
    for a, b in zip(got, oracle_state(ref["state"])):
        assert rel_l2(a, b) <= 1e-5
    assert abs(J.item() - ref["J"]) <= 1e-5 * abs(ref["J"])
    adj = [a.double().cpu().numpy() for a in s.get_adjoint()[:6]]
    for k in range(6):
        assert rel_l2(adj[k], ref["adjoint"][k]) <= 1e-3, k
    assert rel_l2(grad.double().cpu().numpy(), ref["dJdgamma"]) <= 1e-3


def test_resident_equals_step_path_config2():
    """512 x 256 (the benchmark lattice), FP32: the resident persistent marches and
    the one-launch-per-step kernels give the same gradient (same arithmetic; only
    the compiler's operation fusion may differ)."""
    pb = inputs.config2().with_(n_steps=2000, n_adj=2000)
    g = torch.from_numpy(pb.gamma())
    Ja, ga = LKS(pb, real="f32", path="resident").gradient(g)
    Jb, gb = LKS(pb, real="f32", path="step").gradient(g)
    assert abs(Ja.item() - Jb.item()) <= 1e-6 * abs(Jb.item())
    assert rel_l2(ga.cpu().numpy(), gb.cpu().numpy()) <= 1e-5


@pytest.mark.parametrize("ks", [1, 2, 3])
def test_resident_steps_per_exchange_match_oracle(ks):
    """Resident marches advancing ks steps per exchange of tile bands (temporal
    blocking) on 320 x 130: 32 x 16 tiles with a ragged last tile row two nodes high
    (narrower than the halo of 2 ks), and an odd step count, so that the last
    exchange carries fewer than ks steps."""
    pb = inputs.channel(320, 130, Re=40.0, seed=4, sigma=3.0, strip=3, n_steps=301, n_adj=301)
    g = pb.gamma()
    s = LKS(pb, real="f32", path="resident", res_steps=ks)
    J, grad = s.gradient(torch.from_numpy(g))
    q = s.query()
    assert q.fwd_path == 2 and q.adj_path == 2 and q.device_status == 0
    assert q.res_steps_fwd == ks and q.res_steps_adj == ks
    ref = O.steady_gradient(pb, g)
    got, _ = gpu_state(s)
    for a, b in zip(got, oracle_state(ref["state"])):
        assert rel_l2(a, b) <= 1e-5
    assert abs(J.item() - ref["J"]) <= 1e-5 * abs(ref["J"])
    adj = [a.double().cpu().numpy() for a in s.get_adjoint()[:6]]
    for k in range(6):
        assert rel_l2(adj[k], ref["adjoint"][k]) <= 1e-3, k
    assert rel_l2(grad.double().cpu().numpy(), ref["dJdgamma"]) <= 1e-3


@pytest.mark.parametrize("ks", [2, 3])
def test_resident_steps_per_exchange_config2(ks):
    """512 x 256 (the benchmark lattice, 64 x 16 tiles): ks steps per exchange give
    the gradient of one step per exchange (the per-node arithmetic is the same)."""
    pb = inputs.config2().with_(n_steps=2001, n_adj=2001)
    g = torch.from_numpy(pb.gamma())
    a = LKS(pb, real="f32", path="resident", res_steps=ks)
    Ja, ga = a.gradient(g)
    Jb, gb = LKS(pb, real="f32", path="resident", res_steps=1).gradient(g)
    assert a.query().res_steps_fwd == ks and a.query().res_steps_adj == ks
    assert abs(Ja.item() - Jb.item()) <= 1e-6 * abs(Jb.item())
    assert rel_l2(ga.cpu().numpy(), gb.cpu().numpy()) <= 1e-5


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_waits_give_up_and_report(which):
    """Failure detection without a GPU fault: a device wait on a condition nothing
    satisfies (0: the resident marches' tile flag, 1: the TMA kernels' mbarrier)
    gives up after its iteration limit, records LKS_ERR_TIMEOUT, and the context
    stays usable for the next gradient."""
    import time
    from paper_2411_03090_gb300 import lks
    t0 = time.time()
    assert lks.selftest_wait(which) == 6
    assert time.time() - t0 < 60
    pb = small()
    s = LKS(pb, real="f32")
    J, grad = s.gradient(torch.from_numpy(pb.gamma()))
    assert s.query().device_status == 0 and np.isfinite(J.item())


def test_sensitivity_zero_on_edges_and_finite():
    pb = small()
    s = LKS(pb, real="f32")
    _, grad = s.gradient(torch.from_numpy(pb.gamma()))
    gr = grad.cpu().numpy()
    assert np.all(np.isfinite(gr))
    assert np.all(gr[0, :] == 0) and np.all(gr[-1, :] == 0)
    assert np.all(gr[:, 0] == 0) and np.all(gr[:, -1] == 0)


# ---------------------------------------------------------------------------------------
# Unsteady: plain trajectory and recomputation checkpoints
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("real,tol", [("f64", 1e-10), ("f32", 1e-3)])
def test_unsteady_plain_matches_oracle(real, tol):
    pb = small(steady=False, n_steps=200)
    g = pb.gamma()
    s = LKS(pb, real=real, checkpoint_every=0)
    J, grad = s.gradient(torch.from_numpy(g))
    ref = O.unsteady_gradient(pb, g)
    assert abs(J.item() - ref["J"]) <= (1e-11 if real == "f64" else 1e-5) * abs(ref["J"])
    assert rel_l2(grad.double().cpu().numpy(), ref["dJdgamma"]) <= tol


@pytest.mark.parametrize("K", [1, 37, 64, 200, 500])
def test_checkpoint_f32_snapshots_equal_plain(K):
    """Recomputation from FP32 snapshots reproduces the stored trajectory exactly, so
    the gradient equals the plain form bit for bit (any K, ragged last segment)."""
    pb = small(steady=False, n_steps=200)
    g = torch.from_numpy(pb.gamma())
    J0, g0 = LKS(pb, real="f32", checkpoint_every=0).gradient(g)
    J1, g1 = LKS(pb, real="f32", checkpoint_every=K, snapshot="f32").gradient(g)
    assert J0.item() == J1.item()
    assert torch.equal(g0, g1)


def test_checkpoint_overlap_repeated_gradients_on_one_handle():
    """The recompute of a segment runs on the handle's second stream while the
    adjoint marches the next segment; three gradients in a row on one handle (its
    stream and events reused, a different design in between) each equal the plain
    form bit for bit."""
    pb = small(steady=False, n_steps=180, nx=136)
    ga = torch.from_numpy(pb.gamma())
    gb = torch.from_numpy(inputs.channel(136, 40, Re=10.0, seed=9, sigma=2.0, strip=2, n_steps=180,
                                         steady=False, pulse_mean=0.75, pulse_amp=0.25,
                                         pulse_period=120.0).gamma())
    plain = LKS(pb, real="f32", checkpoint_every=0)
    ck = LKS(pb, real="f32", checkpoint_every=25, snapshot="f32")
    for g in (ga, gb, ga):
        J0, g0 = plain.gradient(g)
        J1, g1 = ck.gradient(g)
        assert J0.item() == J1.item()
        assert torch.equal(g0, g1)


@pytest.mark.parametrize("nx", [70, 136])
@pytest.mark.parametrize("K", [20, 50])
@pytest.mark.parametrize("snap", ["bf16", "f16"])
def test_checkpoint_reduced_snapshots_match_oracle(snap, K, nx):
    """BF16 / FP16 snapshots with per-field scaling, segments recomputed in FP32:
    the gradient is within 1e-3 relative L2 of the FP64 oracle's (the gradient
    tolerance of the FP32 path; measured 1.8e-4 to 2.7e-4 with BF16, 3e-5 to 5e-5
    with FP16), and J, which the forward march computes before any snapshot is
    read, within 1e-5.  nx = 136 runs the TMA-staged kernels."""
    pb = small(steady=False, n_steps=200, nx=nx)
    g = pb.gamma()
    ref = O.unsteady_gradient(pb, g)
    J1, g1 = LKS(pb, real="f32", checkpoint_every=K, snapshot=snap).gradient(torch.from_numpy(g))
    assert abs(J1.item() - ref["J"]) <= 1e-5 * abs(ref["J"])
    assert rel_l2(g1.double().cpu().numpy(), ref["dJdgamma"]) <= 1e-3


def test_natural_convection_cavity_on_the_gpu():
    """Sec. 2.6's natural-convection check (closed cavity, heated bottom segment,
    Boussinesq force, K_s = 10 K_f; `inputs.natural_convection_cavity`) on the FP64
    GPU path: after 46000 forward and 40000 adjoint steps the gradient equals the
    oracle's to 1e-9, and ALKS agrees in direction (cosine >= 0.99) with central
    differences of J computed on the GPU by tolerance marches warm-started from the
    converged state."""
    pb, g = inputs.natural_convection_cavity(0.5)
    pb = pb.with_(n_steps=46000, n_adj=40000)
    s = LKS(pb, real="f64")
    J, grad = s.gradient(torch.from_numpy(g))
    assert s.query().device_status == 0
    ref = O.steady_gradient(pb, g)
    assert abs(J.item() - ref["J"]) <= 1e-11 * abs(ref["J"])
    gr = grad.cpu().numpy()
    assert rel_l2(gr, ref["dJdgamma"]) <= 1e-9
    w = LKS(pb.with_(n_steps=1000), real="f64", tol=1e-13, max_steps=400000, warm_start=True)
    gt = torch.from_numpy(g)
    w.lks_forward(gt)
    base = [x.clone() for x in w.get_state()]
    j, eps = pb.ny // 2, 1e-3
    a, b = [], []
    for i in (20, 28, 36, 44, 52):
        v = []
        for sg in (1, -1):
            gg = g.copy()
            gg[j, i] += sg * eps
            w.set_state(gt, base[0], base[1], base[2], base[3])
            v.append(w.lks_forward(torch.from_numpy(gg)).item())
        a.append(gr[j, i])
        b.append((v[0] - v[1]) / (2 * eps))
    a, b = np.array(a), np.array(b)
    assert a @ b / np.linalg.norm(a) / np.linalg.norm(b) >= 0.99, a / b


def _energy_loss_geometry(nx=31, steps=4000, **kw):
    """The 31 x 31 check geometry of Sec. 2.6 (inlet and outlet over rows 10..20,
    nu = 0.1, gamma = 0.1 in the centre circle of radius 5, 0.9 elsewhere) with the
    energy loss in J; nx = 32 adds a column so that FP32 would take the per-tile TMA
    kernels, which do not carry the energy loss, without the step-kernel gate."""
    n, nu = 31, 0.1
    pb = inputs.Problem(nx=nx, ny=n, nu=nu, alpha_bar=1e3 * nu, u_max=nu / 10.0, in_y0=10, in_y1=20,
                        out_y0=10, out_y1=20, n_steps=steps, n_adj=steps, kappa_E=1.0, **kw)
    yy, xx = np.mgrid[0:n, 0:nx]
    return pb, np.where((xx - 15) ** 2 + (yy - 15) ** 2 <= 25.0, 0.1, 0.9)


@pytest.mark.parametrize("nx", [31, 32])
@pytest.mark.parametrize("real,jtol,gtol", [("f64", 1e-12, 1e-9), ("f32", 1e-5, 2e-3)])
def test_energy_loss_steady_matches_oracle(real, jtol, gtol, nx):
    """Energy loss (Eq. objective_doublepipe, kappa_E = 1) on the check geometry,
    steady, 4000 + 4000 steps: J (dissipation + energy loss) and dJ/dgamma equal the
    oracle's (FP64 to round-off; FP32 within its rounding), and the march ran on the
    per-step kernels."""
    pb, g = _energy_loss_geometry(nx)
    s = LKS(pb, real=real)
    J, grad = s.gradient(torch.from_numpy(g))
    q = s.query()
    assert q.device_status == 0 and q.fwd_path == 1 and q.adj_path == 1
    ref = O.steady_gradient(pb, g)
    assert abs(J.item() - ref["J"]) <= jtol * abs(ref["J"])
    assert rel_l2(grad.double().cpu().numpy(), ref["dJdgamma"]) <= gtol
    # the energy loss's share is not negligible: without it J and the gradient move
    r0 = O.steady_gradient(pb.with_(kappa_E=0.0), g)
    assert rel_l2(r0["dJdgamma"], ref["dJdgamma"]) > 10 * gtol


@pytest.mark.parametrize("real,jtol,gtol", [("f64", 1e-11, 1e-9), ("f32", 1e-5, 2e-3)])
def test_energy_loss_unsteady_matches_oracle(real, jtol, gtol):
    """The time integral of the energy loss under a pulsing inlet (u_in(t) = u_max
    sin(2 pi t / 400), 1200 steps from rest, nx = 32): J summed over levels 1..n and
    the unsteady gradient equal the oracle's."""
    pb, g = _energy_loss_geometry(32, 1200, steady=False, pulse_mean=0.0, pulse_amp=1.0, pulse_period=400.0)
    s = LKS(pb, real=real)
    J, grad = s.gradient(torch.from_numpy(g))
    assert s.query().device_status == 0
    ref = O.unsteady_gradient(pb, g)
    assert abs(J.item() - ref["J"]) <= jtol * abs(ref["J"])
    assert rel_l2(grad.double().cpu().numpy(), ref["dJdgamma"]) <= gtol


def test_energy_loss_gradient_agrees_with_central_differences_on_the_gpu():
    """Steady energy loss on the 31 x 31 check geometry (FP64 GPU path): the J_E share
    of the gradient (kappa_E = 1 minus 0) against central differences of J_E computed
    on the GPU (tolerance marches warm-started from the converged state), along the
    centre line: ratios 0.75..1.1, as the oracle pin finds."""
    pb, g = _energy_loss_geometry(31, 25000)
    _, g1 = LKS(pb, real="f64").gradient(torch.from_numpy(g))
    _, g0 = LKS(pb.with_(kappa_E=0.0), real="f64").gradient(torch.from_numpy(g))
    adj = (g1 - g0).cpu().numpy()
    w = [LKS(pb.with_(n_steps=1000, kappa_E=ke), real="f64", tol=1e-15, max_steps=400000, warm_start=True)
         for ke in (1.0, 0.0)]
    gt = torch.from_numpy(g)
    w[0].lks_forward(gt)
    base = [x.clone() for x in w[0].get_state()]
    eps = 1e-3
    for i in (6, 10, 15, 21, 25):
        v = []
        for sg in (1, -1):
            gg = torch.from_numpy(g.copy())
            gg[15, i] += sg * eps
            jj = []
            for h in w:
                h.set_state(gt, base[0], base[1], base[2])
                jj.append(h.lks_forward(gg).item())
            v.append(jj[0] - jj[1])
        fd = (v[0] - v[1]) / (2 * eps)
        assert 0.75 <= adj[15, i] / fd <= 1.1, (i, adj[15, i], fd)


def test_forced_convection_check_on_the_gpu():
    """Sec. 2.6's forced-convection check (`inputs.forced_convection_check`: T fixed on
    the inlet edge, adiabatic elsewhere, heat source Q = beta_gamma (1 - T) and the
    heat-exchange objective) on the FP64 GPU path: after 40000 + 40000 steps J and
    the gradient equal the oracle's to 1e-11 and 1e-9; the heat-exchange share of the
    gradient (kappa_Q = 1 minus kappa_Q = 0) agrees with central differences of that
    share computed on the GPU (tolerance marches warm-started from the converged
    state) along the centre line: cosine >= 0.999, ratios 0.8..1.05, as the oracle
    pin finds."""
    pb, g = inputs.forced_convection_check()
    s1 = LKS(pb, real="f64")
    J1, g1 = s1.gradient(torch.from_numpy(g))
    assert s1.query().device_status == 0
    ref = O.steady_gradient(pb, g)
    assert abs(J1.item() - ref["J"]) <= 1e-11 * abs(ref["J"])
    assert rel_l2(g1.cpu().numpy(), ref["dJdgamma"]) <= 1e-9
    s0 = LKS(pb.with_(kappa_Q=0.0), real="f64")
    _, g0 = s0.gradient(torch.from_numpy(g))
    sens = (g1 - g0).cpu().numpy()
    gt = torch.from_numpy(g)
    w = [LKS(pb.with_(n_steps=1000, kappa_Q=kq), real="f64", tol=1e-13, max_steps=400000, warm_start=True)
         for kq in (1.0, 0.0)]
    w[0].lks_forward(gt)
    base = [x.clone() for x in w[0].get_state()]
    j, eps = 15, 1e-3
    a, b = [], []
    for i in (6, 10, 15, 21, 25):
        v = []
        for sg in (1, -1):
            gg = torch.from_numpy(g.copy())
            gg[j, i] += sg * eps
            jq = []
            for h in w:
                h.set_state(gt, base[0], base[1], base[2], base[3])
                jq.append(h.lks_forward(gg).item())
            v.append(jq[0] - jq[1])
        a.append(sens[j, i])
        b.append((v[0] - v[1]) / (2 * eps))
    a, b = np.array(a), np.array(b)
    assert a @ b / np.linalg.norm(a) / np.linalg.norm(b) >= 0.999, a / b
    assert np.all((a / b > 0.8) & (a / b < 1.05)), a / b


@pytest.mark.parametrize("thermal", [False, True])
@pytest.mark.parametrize("K,snap", [(0, "f32"), (50, "bf16"), (37, "f32")])
@pytest.mark.parametrize("seg", ["bf16", "f16"])
def test_16bit_stored_levels_match_oracle(seg, K, snap, thermal):
    """segment_type BF16 / F16: the levels of u, v (and T) that the adjoint reads --
    the whole trajectory (K = 0) or the recomputed segment -- stored in 16 bits
    (packed after each forward step, unpacked before each adjoint step).  J is
    untouched (the forward march computes it) and the gradient stays within 1e-3 of
    the FP64 oracle's; on the TMA-staged kernels (nx = 136), flow and thermal."""
    pb = (thermal_small(False, nx=136) if thermal else small(steady=False, n_steps=200, nx=136))
    g = pb.gamma()
    ref = O.unsteady_gradient(pb, g)
    s = LKS(pb, real="f32", checkpoint_every=K, snapshot=snap, segment=seg)
    J, grad = s.gradient(torch.from_numpy(g))
    assert s.query().device_status == 0
    assert abs(J.item() - ref["J"]) <= 1e-5 * abs(ref["J"])
    assert rel_l2(grad.double().cpu().numpy(), ref["dJdgamma"]) <= 1e-3
    full = LKS(pb, real="f32", checkpoint_every=K, snapshot=snap)
    assert s.workspace.numel() < full.workspace.numel()


# ---------------------------------------------------------------------------------------
# API behaviour
# ---------------------------------------------------------------------------------------
def test_warm_start_continues_the_march():
    """warm_start = 1: a second lks_forward continues from the state the first one
    left, and a second alks_adjoint from its adjoint fields, so two calls of n steps
    equal one call of 2n steps bit for bit (the same kernels run in the same order)."""
    pb = small(n_steps=150, n_adj=120)
    g = torch.from_numpy(pb.gamma())
    a = LKS(pb, real="f64", path="step", warm_start=True)
    a.lks_forward(g)
    Ja = a.lks_forward(g).item()
    a.alks_adjoint()
    a.alks_adjoint()
    ga = a.lks_sensitivity()
    b = LKS(pb.with_(n_steps=300, n_adj=240), real="f64", path="step")
    Jb = b.lks_forward(g).item()
    b.alks_adjoint()
    gb = b.lks_sensitivity()
    assert Ja == Jb
    for x, y in zip(a.get_state()[:3], b.get_state()[:3]):
        assert torch.equal(x, y)
    assert torch.equal(ga, gb)
    assert a.query().forward_steps == 300 and a.query().adjoint_steps == 240


def test_gpu_gradient_agrees_with_central_differences():
    """Sec. 2.6 verification on the GPU path (FP64 instance): a converged steady
    porous channel, ALKS sensitivity against central differences of J with step
    1e-4 (Eq. sensfdm) on 12 design nodes drawn with seed 22 at least 3 nodes from
    an edge.  Each perturbed march is a tolerance march warm-started from the
    converged state of the unperturbed design.  ALKS is a continuous adjoint with
    approximate edge rules, so the check is on direction: cosine >= 0.99."""
    pb = inputs.Problem(nx=40, ny=24, nu=0.1, alpha_bar=100.0, u_max=0.05, sigma=2.0, strip=2, seed=7,
                        n_steps=2000, n_adj=2000)
    g = pb.gamma()
    s = LKS(pb, real="f64", tol=1e-14, max_steps=400000, warm_start=True)
    gt = torch.from_numpy(g)
    J0, grad = s.gradient(gt)
    grad = grad.cpu().numpy()
    base = [x.clone() for x in s.get_state()]
    rng = np.random.default_rng(22)
    cand = [(j, i) for j in range(3, pb.ny - 3) for i in range(3, pb.nx - 3)]
    nodes = [cand[k] for k in rng.choice(len(cand), 12, replace=False)]
    eps = 1e-4
    fd, ad = [], []
    for (j, i) in nodes:
        Js = []
        for sgn in (1.0, -1.0):
            gp = g.copy()
            gp[j, i] += sgn * eps
            s.set_state(gt, base[0], base[1], base[2])
            Js.append(s.lks_forward(torch.from_numpy(gp)).item())
            assert s.query().fwd_change <= 1e-14
        fd.append((Js[0] - Js[1]) / (2 * eps))
        ad.append(grad[j, i])
    fd, ad = np.array(fd), np.array(ad)
    cos = fd @ ad / np.linalg.norm(fd) / np.linalg.norm(ad)
    assert cos >= 0.99, (cos, ad / fd)


@pytest.mark.parametrize("real,path,nx,ftol,gtol", [("f64", "step", 70, 1e-11, 1e-10), ("f32", "step", 136, 1e-5, 1e-3),
                                                    ("f32", "resident", 136, 1e-5, 1e-3),
                                                    ("f32", "column", 136, 1e-5, 1e-3)])
def test_pressure_drop_objective_matches_oracle(real, path, nx, ftol, gtol):
    """J = J_O + J_p with the static pressure drop (Eq. objective_pipebend, kappa_p = 1)
    on a channel whose inlet covers rows 8..30 of the left edge (walls elsewhere on it)
    and whose outlet covers rows 5..34: J and the adjoint fields (which carry the
    boundary objective term of Eqs. afboundaryu / afboundaryp) and dJ/dgamma against
    the oracle, on the per-step (plain and TMA-staged), resident and warp-column
    kernels."""
    pb = small(nx=nx, kappa_p=1.0, in_y0=8, in_y1=30, out_y0=5, out_y1=34)
    g = pb.gamma()
    s = LKS(pb, real=real, path=path)
    J, grad = s.gradient(torch.from_numpy(g))
    q = s.query()
    assert q.device_status == 0 and q.fwd_path == {"step": 1, "resident": 2, "column": 3}[path]
    ref = O.steady_gradient(pb, g)
    assert abs(O.pressure_drop(pb, ref["state"])) > 1e-3 * abs(ref["J"])  # the term matters
    assert abs(J.item() - ref["J"]) <= ftol * abs(ref["J"])
    adj = [a.double().cpu().numpy() for a in s.get_adjoint()[:6]]
    for k in range(6):
        assert rel_l2(adj[k], ref["adjoint"][k]) <= gtol, k
    assert rel_l2(grad.double().cpu().numpy(), ref["dJdgamma"]) <= gtol


def test_pressure_drop_verification_of_the_paper_on_the_gpu():
    """Sec. 2.6's pressure-drop verification on the GPU path (FP64 instance), 31 x 31
    nodes: walls, inlet and outlet over rows 10..20, nu = 0.1, Re = 1 on the length 10,
    gamma = 0.1 in the centre circle of radius 5 and 0.9 elsewhere, J = J_p.  The
    gradient equals the oracle's to 1e-10, and ALKS agrees with central differences of
    J (eps = 1e-3, tolerance marches warm-started from the converged state) along the
    centre line within 0.75..1.1, as the oracle pin finds."""
    n, nu = 31, 0.1
    pb = inputs.Problem(nx=n, ny=n, nu=nu, alpha_bar=1e3 * nu, u_max=nu / 10.0, in_y0=10, in_y1=20,
                        out_y0=10, out_y1=20, n_steps=25000, n_adj=25000)
    yy, xx = np.mgrid[0:n, 0:n]
    g = np.where((xx - 15) ** 2 + (yy - 15) ** 2 <= 25.0, 0.1, 0.9)
    # J_p alone: the dissipation's share is removed by differencing kappa_p = 1 and 0
    s1 = LKS(pb.with_(kappa_p=1.0), real="f64")
    s0 = LKS(pb, real="f64")
    J1, g1 = s1.gradient(torch.from_numpy(g))
    J0, g0 = s0.gradient(torch.from_numpy(g))
    adj = (g1 - g0).cpu().numpy()
    r1 = O.steady_gradient(pb.with_(kappa_p=1.0), g)
    r0 = O.steady_gradient(pb, g)
    assert rel_l2(adj, r1["dJdgamma"] - r0["dJdgamma"]) <= 1e-9
    st = LKS(pb.with_(n_steps=500), real="f64", tol=1e-15, max_steps=400000, warm_start=True)
    gt = torch.from_numpy(g)
    st.lks_forward(gt)
    base = [x.clone() for x in st.get_state()]
    eps = 1e-3
    for i in (6, 15, 21):
        v = []
        for sg in (1, -1):
            gg = g.copy()
            gg[15, i] += sg * eps
            st.set_state(gt, base[0], base[1], base[2])
            st.lks_forward(torch.from_numpy(gg))
            d = st.get_state()[0].cpu().numpy()  # rho - 1
            v.append((d[10:21, 0].sum() - d[10:21, -1].sum()) / 3.0)  # J_p (the 1s cancel)
        fd = (v[0] - v[1]) / (2 * eps)
        assert 0.75 <= adj[15, i] / fd <= 1.1, (i, adj[15, i], fd)


def thermal_sources_case(steady, nx, **kw):
    """Thermal channel with a heat source Q = beta_gamma (1 - T) (beta_bar = 0.05), the
    heat-exchange objective (kappa_Q = 0.5) and a Boussinesq force (g beta = (0,
    -2e-3), T_ref = 0.5): a heated bottom wall drives buoyancy."""
    base = dict(beta_bar=0.05, q_beta=0.1, kappa_Q=0.5, gb_x=0.0, gb_y=-2e-3, T_ref=0.5)
    base.update(kw)
    return thermal_small(steady, nx=nx, **base)


@pytest.mark.parametrize("steady", [True, False])
@pytest.mark.parametrize("real,nx,jtol,gtol", [("f64", 70, 1e-11, 1e-10), ("f32", 136, 1e-5, 1e-3)])
def test_heat_source_and_boussinesq_match_oracle(steady, real, nx, jtol, gtol):
    """Heat source (Eqs. heatsource, betagamma), heat-exchange objective (Eq.
    objective_heatexchanger) and Boussinesq force (Eq. boussinesqforce) on the
    per-step kernels (plain FP64, TMA-staged FP32): J, the nine adjoint fields and
    dJ/dgamma against the oracle, steady and unsteady."""
    pb = thermal_sources_case(steady, nx)
    g = pb.gamma()
    s = LKS(pb, real=real)
    J, grad = s.gradient(torch.from_numpy(g))
    q = s.query()
    assert q.device_status == 0 and q.fwd_path == 1 and q.adj_path == 1
    ref = O.steady_gradient(pb, g) if steady else O.unsteady_gradient(pb, g)
    assert abs(J.item() - ref["J"]) <= jtol * abs(ref["J"])
    if steady:
        adj = [a.double().cpu().numpy() for a in s.get_adjoint()]
        for k in range(9):
            assert rel_l2(adj[k], ref["adjoint"][k]) <= gtol, k
    assert rel_l2(grad.double().cpu().numpy(), ref["dJdgamma"]) <= gtol
    # the source terms matter: without them the gradient differs by far more than gtol
    plain = O.steady_gradient(pb.with_(beta_bar=0.0, kappa_Q=0.0, gb_y=0.0), g) if steady else \
        O.unsteady_gradient(pb.with_(beta_bar=0.0, kappa_Q=0.0, gb_y=0.0), g)
    assert rel_l2(plain["dJdgamma"], ref["dJdgamma"]) > 100 * gtol


def test_thermal_sources_reject_the_resident_and_column_paths():
    pb = thermal_sources_case(True, 136)
    for path in ("resident", "column"):
        with pytest.raises(LKSError):
            LKS(pb, real="f32", path=path)


def test_gradient_host_matches_device():
    pb = small()
    g = pb.gamma()
    s = LKS(pb, real="f32")
    J, grad = s.gradient(torch.from_numpy(g))
    Jh, gh = s.gradient_host(g)
    assert Jh == J.item()
    np.testing.assert_array_equal(gh, grad.cpu().numpy())


def test_autograd_function():
    pb = small()
    s = LKS(pb, real="f64")
    gam = torch.from_numpy(pb.gamma()).cuda().requires_grad_(True)
    J = objective(gam, s)
    (2.0 * J).backward()
    ref = O.steady_gradient(pb, pb.gamma())
    assert rel_l2(gam.grad.cpu().numpy(), 2.0 * ref["dJdgamma"]) <= 1e-10


def test_call_order_and_unstable_status():
    pb = small()
    s = LKS(pb, real="f32")
    with pytest.raises(LKSError) as e:
        s.alks_adjoint()
    assert e.value.status == 7
    # an inlet above the |u| <= 0.5 bound is reported through the device status word
    bad = small(n_steps=5).with_(u_max=0.7)
    sb = LKS(bad, real="f32")
    sb.lks_forward(torch.from_numpy(bad.gamma()))
    st = sb.query()
    assert st.device_status == 4


# ---------------------------------------------------------------------------------------
# Thermal lattice (T-fixed inlet and heated bottom wall, adiabatic top and outlet)
# ---------------------------------------------------------------------------------------
def thermal_small(steady, nx=70, **kw):
    base = dict(seed=3, sigma=2.0, strip=2, n_steps=200, n_adj=200, thermal=1, kappa_T=1e-2,
                t_kind=[0, 1, 0, 1], t_val=[0.0, 0.0, 1.0, 0.0])
    base.update(kw)
    if not steady:
        base.update(steady=False, pulse_mean=0.75, pulse_amp=0.25, pulse_period=120.0)
    p = inputs.channel(nx, 40, Re=10.0, **base)
    p.K_f = p.nu / 0.71
    p.K_s = p.K_f
    return p


def thermal_column_case(steady=True):
    """200 x 150 thermal channel with fixed-T and heat-flux edges: interior and edge
    column tiles (60 x 40) for the flow and the temperature kernels."""
    base = dict(seed=3, sigma=3.0, strip=3, n_steps=200, n_adj=200, thermal=1, kappa_T=1e-2,
                t_kind=[0, 1, 0, 1], t_val=[0.0, 0.0, 1.0, 0.0])
    if not steady:
        base.update(steady=False, pulse_mean=0.75, pulse_amp=0.25, pulse_period=90.0, n_steps=120)
    p = inputs.channel(200, 150, Re=60.0, **base)
    p.K_f = p.nu / 0.71
    p.K_s = p.K_f
    return p


@pytest.mark.parametrize("steady", [True, False])
def test_thermal_column_forward_equals_tma_step_bitwise(steady):
    """The warp-column forward (flow kernel, then the temperature kernel) computes
    every node with the arithmetic of the thermal TMA kernel: identical states,
    adjoints and gradients; J differs only in the grouping of its FP64 sums."""
    pb = thermal_column_case(steady)
    g = torch.from_numpy(pb.gamma())
    K = 0 if steady else 20
    a = LKS(pb, real="f32", path="column", checkpoint_every=K)
    b = LKS(pb, real="f32", path="step", checkpoint_every=K)
    Ja, ga = a.gradient(g)
    Jb, gb = b.gradient(g)
    assert a.query().fwd_path == 3 and b.query().fwd_path == 1
    for x, y in zip(a.get_state(), b.get_state()):
        assert torch.equal(x, y)
    for x, y in zip(a.get_adjoint(), b.get_adjoint()):
        assert torch.equal(x, y)
    assert torch.equal(ga, gb)
    assert abs(Ja.item() - Jb.item()) <= 1e-12 * abs(Jb.item())


def test_thermal_column_forward_matches_oracle():
    pb = thermal_column_case(True)
    g = pb.gamma()
    s = LKS(pb, real="f32", path="column")
    J = s.lks_forward(torch.from_numpy(g)).item()
    assert s.query().fwd_path == 3 and s.query().device_status == 0
    st, _, _, _ = O.forward(pb, g, pb.n_steps)
    got, T = gpu_state(s)
    for x, y in zip(got, oracle_state(st)):
        assert rel_l2(x, y) <= 1e-5
    assert rel_l2(T, st.T) <= 1e-5
    assert abs(J - O.objective(pb, g, st)) <= 1e-4 * abs(J)


@pytest.mark.parametrize("path", ["step", "resident"])
@pytest.mark.parametrize("real,tol", [("f64", 1e-11), ("f32", 1e-5)])
def test_thermal_forward_matches_oracle(real, tol, path):
    pb = thermal_small(True)
    g = pb.gamma()
    s = LKS(pb, real=real, path=path)
    J = s.lks_forward(torch.from_numpy(g)).item()
    st, _, _, _ = O.forward(pb, g, pb.n_steps)
    got, T = gpu_state(s)
    for a, b in zip(got, oracle_state(st)):
        assert rel_l2(a, b) <= tol
    assert rel_l2(T, st.T) <= tol
    assert abs(J - O.objective(pb, g, st)) <= 10 * tol * abs(J)


def test_single_steps_full_size_config3():
    """1024 x 512 thermal unsteady channel (config 3), FP32, the per-step TMA kernels
    the benchmark runs: one forward step from a developed state (the oracle's after
    300 steps, rounded to FP32) and one ALKS step from seeded adjoint fields equal
    the oracle's steps from the same fields (all nine adjoint fields)."""
    pb = inputs.config3()
    g = pb.gamma()
    gf = f32(g)
    st = oracle_developed_state(pb, g, 300)
    s = LKS(pb, real="f32")
    set_gpu_state(s, g, st, 300)
    d0 = st.rho - 1.0
    s.march(1)
    assert s.query().fwd_path == 1 and s.query().device_status == 0
    (d1, u1, v1), T1 = gpu_state(s)
    ref = O.forward_step(pb, gf, 301, st)
    for a, b, scale in ((d1, ref.rho - 1.0, np.abs(d0).max()), (u1, ref.u, pb.u_max),
                        (v1, ref.v, pb.u_max), (T1, ref.T, 1.0)):
        assert np.abs(a - b).max() <= 2e-6 * scale
    # ALKS step with the state frozen at the oracle's level 301 (rounded to FP32)
    st1 = O.State(pb.ny, pb.nx)
    st1.rho, st1.u, st1.v, st1.T = 1.0 + f32(ref.rho - 1.0), f32(ref.u), f32(ref.v), f32(ref.T)
    set_gpu_state(s, g, st1, 301)
    rng = np.random.default_rng(7)
    a0 = f32(1e-3 * rng.standard_normal((9, pb.ny, pb.nx)))
    s.set_adjoint([torch.from_numpy(np.ascontiguousarray(a0[q])) for q in range(9)])
    s.adjoint_march(1)
    a1 = [a.double().cpu().numpy() for a in s.get_adjoint()]
    ref_a = O.adjoint_step(pb, gf, st1, st1, a0)
    for q in range(9):
        scale = np.abs(ref_a[q]).max()
        assert np.abs(a1[q] - ref_a[q]).max() <= 1e-5 * scale, q


@pytest.mark.parametrize("real,tol", [("f64", 1e-10), ("f32", 1e-3)])
def test_thermal_steady_gradient_matches_oracle(real, tol):
    pb = thermal_small(True)
    g = pb.gamma()
    s = LKS(pb, real=real)
    J, grad = s.gradient(torch.from_numpy(g))
    ref = O.steady_gradient(pb, g)
    adj = [a.double().cpu().numpy() for a in s.get_adjoint()]
    for q in range(9):
        assert rel_l2(adj[q], ref["adjoint"][q]) <= tol, q
    assert rel_l2(grad.double().cpu().numpy(), ref["dJdgamma"]) <= tol


@pytest.mark.parametrize("real,tol", [("f64", 1e-10), ("f32", 1e-3)])
def test_thermal_unsteady_gradient_matches_oracle(real, tol):
    """Unsteady thermal problem with a conductivity contrast (K_s = 2 K_f), so the
    B'(gamma) grad T . q~ term of the sensitivity is exercised."""
    pb = thermal_small(False, n_steps=150)
    pb.K_s = 2.0 * pb.K_f
    g = pb.gamma()
    s = LKS(pb, real=real, checkpoint_every=0)
    J, grad = s.gradient(torch.from_numpy(g))
    ref = O.unsteady_gradient(pb, g)
    assert abs(J.item() - ref["J"]) <= (1e-11 if real == "f64" else 1e-5) * abs(ref["J"])
    assert rel_l2(grad.double().cpu().numpy(), ref["dJdgamma"]) <= tol


def test_thermal_checkpoints_equal_plain():
    pb = thermal_small(False, n_steps=150)
    g = torch.from_numpy(pb.gamma())
    J0, g0 = LKS(pb, real="f32", checkpoint_every=0).gradient(g)
    J1, g1 = LKS(pb, real="f32", checkpoint_every=40, snapshot="f32").gradient(g)
    assert J0.item() == J1.item()
    assert torch.equal(g0, g1)



# ---------------------------------------------------------------------------------------
# TMA-staged per-step kernels (FP32, nx % 4 == 0)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("path", ["step", "column"])
def test_tma_forward_matches_oracle(path):
    pb = small(nx=136)
    g = pb.gamma()
    s = LKS(pb, real="f32", path=path)
    J = s.lks_forward(torch.from_numpy(g)).item()
    st, _, _, _ = O.forward(pb, g, pb.n_steps)
    got, _ = gpu_state(s)
    for a, b in zip(got, oracle_state(st)):
        assert rel_l2(a, b) <= 1e-5
    assert abs(J - O.objective(pb, g, st)) <= 1e-5 * abs(J)


@pytest.mark.parametrize("path", ["step", "column"])
def test_tma_steady_gradient_matches_oracle(path):
    pb = small(nx=136)
    g = pb.gamma()
    s = LKS(pb, real="f32", path=path)
    J, grad = s.gradient(torch.from_numpy(g))
    ref = O.steady_gradient(pb, g)
    adj = [a.double().cpu().numpy() for a in s.get_adjoint()[:6]]
    for q in range(6):
        assert rel_l2(adj[q], ref["adjoint"][q]) <= 1e-3, q
    assert rel_l2(grad.double().cpu().numpy(), ref["dJdgamma"]) <= 1e-3


@pytest.mark.parametrize("K,path", [(0, "auto"), (64, "auto"), (0, "column"), (64, "column")])
def test_tma_unsteady_gradient_matches_oracle(K, path):
    pb = small(steady=False, nx=136, n_steps=200)
    g = pb.gamma()
    s = LKS(pb, real="f32", checkpoint_every=K, path=path)
    J, grad = s.gradient(torch.from_numpy(g))
    ref = O.unsteady_gradient(pb, g)
    assert abs(J.item() - ref["J"]) <= 1e-5 * abs(ref["J"])
    assert rel_l2(grad.double().cpu().numpy(), ref["dJdgamma"]) <= 1e-3


@pytest.mark.parametrize("steady", [True, False])
def test_tma_thermal_gradient_matches_oracle(steady):
    pb = thermal_small(steady, nx=136, n_steps=150)
    if not steady:
        pb.K_s = 2.0 * pb.K_f
    g = pb.gamma()
    s = LKS(pb, real="f32", path="step")
    J, grad = s.gradient(torch.from_numpy(g))
    ref = O.steady_gradient(pb, g) if steady else O.unsteady_gradient(pb, g)
    assert abs(J.item() - ref["J"]) <= 1e-4 * abs(ref["J"])
    assert rel_l2(grad.double().cpu().numpy(), ref["dJdgamma"]) <= 1e-3


# ---------------------------------------------------------------------------------------
# Warp-column kernels (path "column"; chosen automatically on large lattices)
# ---------------------------------------------------------------------------------------
def column_case(steady=True, **kw):
    """200 x 150: interior column tiles (60 x 40 forward, 28 x 32 adjoint) as well as
    edge tiles and ragged last tiles (forward 200 = 3 x 60 + 20, 150 = 3 x 40 + 30;
    adjoint 200 = 7 x 28 + 4)."""
    base = dict(seed=9, sigma=3.0, strip=3, n_steps=300, n_adj=300)
    base.update(kw)
    if not steady:
        base.update(steady=False, pulse_mean=0.75, pulse_amp=0.25, pulse_period=90.0, n_steps=150)
    return inputs.channel(200, 150, Re=60.0, **base)


def test_column_steady_gradient_matches_oracle():
    pb = column_case()
    g = pb.gamma()
    s = LKS(pb, real="f32", path="column")
    J, grad = s.gradient(torch.from_numpy(g))
    q = s.query()
    assert q.fwd_path == 3 and q.adj_path == 3 and q.device_status == 0
    ref = O.steady_gradient(pb, g)
    got, _ = gpu_state(s)
    for a, b in zip(got, oracle_state(ref["state"])):
        assert rel_l2(a, b) <= 1e-5
    assert abs(J.item() - ref["J"]) <= 1e-5 * abs(ref["J"])
    assert rel_l2(grad.double().cpu().numpy(), ref["dJdgamma"]) <= 1e-3


@pytest.mark.parametrize("path", ["step", "column", "auto"])
def test_unsteady_J_every_path_matches_oracle(path):
    """J integrated over the march (Eq. fj, Sec. 2.5) on a 200 x 150 lattice, where the 64 x 8 TMA
    tiles (76) outnumber the 32 x 16 plain tiles (70): every CTA's objective partial
    must land in the partial sums."""
    pb = column_case(False)
    g = pb.gamma()
    s = LKS(pb, real="f32", path=path, checkpoint_every=25)
    J = s.lks_forward(torch.from_numpy(g)).item()
    _, _, _, Jo = O.forward(pb, g, pb.n_steps, accumulate_J=True)
    assert abs(J - Jo) <= 2e-6 * abs(Jo)


def test_exec_path_is_honoured_on_a_large_lattice():
    """2048 x 1024 has more than four column tiles per SM: the automatic choice is
    the warp-column forward, while an explicit step path keeps the per-tile kernels."""
    pb = inputs.roofline2d(2048).with_(ny=1024, n_steps=3, n_adj=3)
    g = torch.from_numpy(pb.gamma())
    paths = {}
    for path in ("auto", "step", "column"):
        s = LKS(pb, real="f32", path=path)
        s.lks_forward(g)
        paths[path] = s.query().fwd_path
    assert paths == {"auto": 3, "step": 1, "column": 3}


@pytest.mark.parametrize("steady", [True, False])
def test_column_equals_tma_step_bitwise(steady):
    """The warp-column kernels compute every node with the arithmetic of the
    per-tile TMA kernels: identical states, adjoints and gradients (J differs
    only in the grouping of its FP64 partial sums)."""
    pb = column_case(steady)
    g = torch.from_numpy(pb.gamma())
    a = LKS(pb, real="f32", path="column", checkpoint_every=0 if steady else 25)
    b = LKS(pb, real="f32", path="step", checkpoint_every=0 if steady else 25)
    Ja, ga = a.gradient(g)
    Jb, gb = b.gradient(g)
    assert a.query().fwd_path == 3 and b.query().fwd_path == 1
    # non-thermal: get_state writes drho, u, v (the T output is left untouched)
    for x, y in zip(a.get_state()[:3], b.get_state()[:3]):
        assert torch.equal(x, y)
    for x, y in zip(a.get_adjoint()[:6], b.get_adjoint()[:6]):
        assert torch.equal(x, y)
    assert torch.equal(ga, gb)
    assert abs(Ja.item() - Jb.item()) <= 1e-12 * abs(Jb.item())
