"""The allocation-free gradient entry point, lks_gradient_noalloc.

Some callers cannot call cudaMalloc and cannot hand the library a workspace (a
plugin whose host application owns all device memory through a fixed pool, or a
latency-critical loop where the implicit synchronisation of cudaMalloc is not
allowed).  For them the library runs the same gradient with its workspace in a
static device array.  These tests call that entry point through the C ABI, twice
in a row (the array keeps the previous call's contents), and compare it with the
handle-based entry points on the same inputs, at the tolerances of the GPU
parity tests.  The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2411_03090_gb300 import LKS, lks  # noqa: E402


def _rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _noalloc(desc, gamma, stream):
    L = lks.load()
    J = torch.zeros((), dtype=torch.float64, device=gamma.device)
    out = torch.empty_like(gamma)
    st = L.lks_gradient_noalloc(C.byref(desc), C.c_void_p(gamma.data_ptr()), C.c_void_p(J.data_ptr()),
                                C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert st == 0, lks.load().lks_status_string(st)
    stream.synchronize()
    return J.item(), out.double().cpu().numpy()


def _case(kind):
    """(problem, real type, checkpoint spacing, snapshot type) of each layout the
    static array can hold: steady and unsteady FP32, FP64, thermal, and an unsteady
    problem with BF16 checkpoints and recomputed segments."""
    pb = inputs.config1().with_(n_steps=400, n_adj=400)
    unsteady = dict(steady=False, pulse_mean=0.75, pulse_amp=0.25, pulse_period=150.0, n_steps=150)
    if kind == "steady":
        return pb, "f32", 0, "f32"
    if kind == "unsteady":
        return pb.with_(**unsteady), "f32", 0, "f32"
    if kind == "f64":
        return pb.with_(nx=40, ny=24, n_steps=200, n_adj=200), "f64", 0, "f32"
    if kind == "thermal":
        th = pb.with_(nx=48, ny=32, thermal=1, kappa_T=1e-2, K_f=0.2, K_s=0.2, t_kind=[0, 1, 0, 1],
                      t_val=[0.0, 0.0, 1.0, 0.0], **unsteady)
        return th, "f32", 0, "f32"
    if kind == "checkpoint_bf16":
        return pb.with_(**unsteady), "f32", 40, "bf16"
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["steady", "unsteady", "f64", "thermal", "checkpoint_bf16"])
def test_noalloc_matches_handle_path_twice(kind):
    pb, real, K, snap = _case(kind)
    dt = torch.float64 if real == "f64" else torch.float32
    g = torch.from_numpy(pb.gamma()).to(dt).cuda()
    s = LKS(pb, real=real, checkpoint_every=K, snapshot=snap)
    J_ref, grad_ref = s.gradient(g)
    J_ref = J_ref.item()
    grad_ref = grad_ref.double().cpu().numpy()
    desc = lks.make_desc(pb, real, checkpoint_every=K, snapshot=snap)
    assert lks.workspace_size(desc) <= 8 << 20
    stream = torch.cuda.current_stream()
    tol_J, tol_g = (1e-12, 1e-10) if real == "f64" else (1e-5, 1e-3)
    for _ in range(2):
        J, grad = _noalloc(desc, g, stream)
        assert abs(J - J_ref) <= tol_J * abs(J_ref)
        assert _rel_l2(grad, grad_ref) <= tol_g
        assert np.all(np.isfinite(grad))


def test_noalloc_reports_device_failure_as_nan():
    """A device-detected failure (here an inlet above the |u| <= 0.5 bound, recorded
    as instability by the kernels) comes back as a NaN objective; the next call on a
    sound problem clears it."""
    bad = inputs.config1().with_(n_steps=5, n_adj=5, u_max=0.7)
    g = torch.from_numpy(bad.gamma()).float().cuda()
    stream = torch.cuda.current_stream()
    J, _ = _noalloc(lks.make_desc(bad, "f32"), g, stream)
    assert np.isnan(J)
    good = inputs.config1().with_(n_steps=50, n_adj=50)
    J, grad = _noalloc(lks.make_desc(good, "f32"), g, stream)
    assert np.isfinite(J) and np.all(np.isfinite(grad))


def test_noalloc_rejects_oversized_problem():
    pb = inputs.config2()
    desc = lks.make_desc(pb, "f32")
    assert lks.workspace_size(desc) > 8 << 20
    g = torch.zeros(pb.ny, pb.nx, dtype=torch.float32, device="cuda")
    J = torch.zeros((), dtype=torch.float64, device="cuda")
    out = torch.empty_like(g)
    st = lks.load().lks_gradient_noalloc(C.byref(desc), C.c_void_p(g.data_ptr()), C.c_void_p(J.data_ptr()),
                                         C.c_void_p(out.data_ptr()), None)
    assert st == 2  # LKS_ERR_WORKSPACE: larger than LKS_NOALLOC_SCRATCH_BYTES
