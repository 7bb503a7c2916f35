"""Python binding of the C ABI in ``include/lks.h`` (argument marshalling only).

Every computation runs in the CUDA kernels of ``_lib/liblks.so``; PyTorch supplies
device memory (the workspace and the caller's buffers) and the CUDA stream.  The
names follow the C entry points: ``lks_forward`` (Steps 2-3 of the paper's
procedure, Sec. 2.7), ``alks_adjoint`` (Step 4), ``lks_sensitivity`` (Step 5).

If the library is missing this module raises; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np
import torch

from . import _build

LKS_DESC_VERSION = 3
STATUS = {0: "ok", 1: "invalid argument", 2: "workspace", 3: "CUDA error", 4: "unstable",
          5: "not converged", 6: "timeout", 7: "calls out of order"}
REAL = {"f32": 0, "f64": 1}
SNAP = {"f32": 0, "bf16": 1, "f16": 2}
PATH = {"auto": 0, "step": 1, "resident": 2, "column": 3}
LATTICE_D3Q19 = 1
N_ADJ_FIELDS_3D = 10
N_ADJ_FIELDS = 9
ADJ_NAMES = ("rho_t", "ux_t", "uy_t", "sxx_t", "sxy_t", "syy_t", "T_t", "qx_t", "qy_t")


class LKSError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: status {status} ({STATUS.get(status, '?')})")
        self.status = status


class Desc(C.Structure):
    """Mirror of ``lks_problem_desc``."""

    _fields_ = [
        ("version", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("real_type", C.c_int32),
        ("nu", C.c_double), ("alpha_bar", C.c_double), ("q_alpha", C.c_double),
        ("u_max", C.c_double), ("pulse_mean", C.c_double), ("pulse_amp", C.c_double),
        ("pulse_period", C.c_double),
        ("in_y0", C.c_int32), ("in_y1", C.c_int32), ("out_y0", C.c_int32), ("out_y1", C.c_int32),
        ("rho_out", C.c_double),
        ("thermal", C.c_int32), ("steady", C.c_int32),
        ("K_f", C.c_double), ("K_s", C.c_double), ("q_K", C.c_double),
        ("t_kind", C.c_int32 * 4), ("t_val", C.c_double * 4),
        ("kappa_T", C.c_double),
        ("n_steps", C.c_int32), ("n_adj", C.c_int32),
        ("checkpoint_every", C.c_int32), ("snapshot_type", C.c_int32),
        ("exec_path", C.c_int32), ("lattice", C.c_int32), ("nz", C.c_int32), ("res_steps", C.c_int32),
        ("kappa_p", C.c_double),
        ("tol", C.c_double), ("max_steps", C.c_int32),
        ("warm_start", C.c_int32), ("segment_type", C.c_int32),
        ("reserved", C.c_int32 * 4),
        ("beta_bar", C.c_double), ("q_beta", C.c_double), ("kappa_Q", C.c_double),
        ("gb", C.c_double * 2), ("T_ref", C.c_double),
        ("heat_x0", C.c_int32), ("heat_x1", C.c_int32), ("heat_q", C.c_double),
        ("kappa_E", C.c_double),
    ]


class Stats(C.Structure):
    _fields_ = [("forward_steps", C.c_int64), ("adjoint_steps", C.c_int64),
                ("kernel_launches", C.c_int64), ("workspace_bytes", C.c_size_t),
                ("device_status", C.c_int32), ("phase", C.c_int32),
                ("fwd_path", C.c_int32), ("adj_path", C.c_int32),
                ("res_steps_fwd", C.c_int32), ("res_steps_adj", C.c_int32),
                ("fwd_change", C.c_double), ("adj_change", C.c_double)]


LKS_BATCH_VERSION = 1
LKS_BATCH_TILE_CONFIGS = 4
TILE_SHAPES = ((64, 8), (32, 16), (128, 4), (64, 16))


class BatchOptions(C.Structure):
    _fields_ = [("version", C.c_int32), ("checkpoint_every", C.c_int32), ("snapshot_type", C.c_int32),
                ("tile_config", C.c_int32), ("use_graph", C.c_int32), ("fwd_column", C.c_int32),
                ("adj_column", C.c_int32), ("reserved", C.c_int32 * 5)]


class BatchStats(C.Structure):
    _fields_ = [("n_designs", C.c_int32), ("tile_config", C.c_int32), ("checkpoint_every", C.c_int32),
                ("n_ckpt", C.c_int32), ("arena_w", C.c_int32), ("arena_h", C.c_int32),
                ("graph", C.c_int32), ("device_status", C.c_int32), ("nodes", C.c_int64),
                ("ntiles", C.c_int64), ("workspace_bytes", C.c_int64), ("kernel_launches", C.c_int64),
                ("gradients", C.c_int64), ("tune_us", C.c_float * LKS_BATCH_TILE_CONFIGS),
                ("fwd_column", C.c_int32), ("tune_fwd_us", C.c_float * LKS_BATCH_TILE_CONFIGS),
                ("tune_col_us", C.c_float), ("adj_column", C.c_int32), ("tune_acol_us", C.c_float)]


# Every symbol the header declares (checked by the CPU test-suite).
EXPORTS = ("lks_workspace_size", "lks_create", "lks_forward", "alks_adjoint", "lks_sensitivity",
           "lks_gradient_host", "lks_set_state", "lks_get_state", "lks_march", "alks_set_adjoint",
           "alks_get_adjoint", "alks_march", "lks_query", "lks_destroy", "lks_status_string",
           "lks_last_error", "lks_edge_moment_map", "lks_edge_objective_map", "lks_selftest_wait",
           "lks_gradient_noalloc",
           "lks_batch_workspace_size", "lks_batch_create", "lks_batch_gradient", "lks_batch_query",
           "lks_batch_destroy", "lks_batch_last_error")

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load ``liblks.so`` (building it first if asked); raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library {_build.LIB} is missing; run __graft_entry__.build()")
    L = C.CDLL(_build.LIB)
    vp, i32, dp = C.c_void_p, C.c_int32, C.POINTER(C.c_double)
    hp = C.c_void_p
    L.lks_workspace_size.argtypes = [C.POINTER(Desc), C.POINTER(C.c_size_t)]
    L.lks_create.argtypes = [C.POINTER(Desc), vp, C.c_size_t, vp, C.POINTER(hp)]
    L.lks_forward.argtypes = [hp, vp, vp]
    L.alks_adjoint.argtypes = [hp]
    L.lks_sensitivity.argtypes = [hp, vp]
    L.lks_gradient_host.argtypes = [hp, vp, vp, vp]
    L.lks_set_state.argtypes = [hp, vp, vp, vp, vp, vp, i32]
    L.lks_get_state.argtypes = [hp, vp, vp, vp, vp]
    L.lks_march.argtypes = [hp, i32]
    L.alks_set_adjoint.argtypes = [hp, C.POINTER(vp)]
    L.alks_get_adjoint.argtypes = [hp, C.POINTER(vp)]
    L.alks_march.argtypes = [hp, i32]
    L.lks_query.argtypes = [hp, C.POINTER(Stats)]
    L.lks_destroy.argtypes = [hp]
    L.lks_status_string.argtypes = [i32]
    L.lks_status_string.restype = C.c_char_p
    L.lks_last_error.argtypes = [hp]
    L.lks_last_error.restype = C.c_char_p
    L.lks_edge_moment_map.argtypes = [C.c_double, i32, dp]
    L.lks_edge_objective_map.argtypes = [C.c_double, i32, dp]
    L.lks_selftest_wait.argtypes = [i32, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]
    L.lks_gradient_noalloc.argtypes = [C.POINTER(Desc), vp, vp, vp, vp]
    L.lks_batch_workspace_size.argtypes = [i32, C.POINTER(Desc), C.POINTER(BatchOptions), C.POINTER(C.c_size_t)]
    L.lks_batch_create.argtypes = [i32, C.POINTER(Desc), C.POINTER(BatchOptions), vp, C.c_size_t, vp,
                                   C.POINTER(hp)]
    L.lks_batch_gradient.argtypes = [hp, C.POINTER(vp), vp, C.POINTER(vp)]
    L.lks_batch_query.argtypes = [hp, C.POINTER(BatchStats)]
    L.lks_batch_destroy.argtypes = [hp]
    L.lks_batch_last_error.argtypes = [hp]
    L.lks_batch_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("lks_status_string", "lks_last_error", "lks_batch_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def make_desc(pb, real: str = "f32", checkpoint_every: int = 0, snapshot: str = "f32",
              path: str = "auto", res_steps: int = 0, tol: float = 0.0, max_steps: int = 0,
              warm_start: bool = False, segment: str = "f32") -> Desc:
    """Descriptor from an ``inputs.Problem``-like object (``inputs.Problem3``: a
    D3Q19 duct).  tol > 0 (steady D2Q9): march to a relative step change of tol,
    at most max_steps steps per march, in chunks of n_steps / n_adj.  warm_start
    (steady D2Q9): each march starts from the handle's current state / adjoint."""
    d = Desc()
    d.version = LKS_DESC_VERSION
    d.nx, d.ny = int(pb.nx), int(pb.ny)
    d.real_type = REAL[real]
    if hasattr(pb, "nz"):
        d.lattice, d.nz = LATTICE_D3Q19, int(pb.nz)
        for name in ("nu", "alpha_bar", "q_alpha", "u_max", "rho_out", "kappa_p"):
            setattr(d, name, float(getattr(pb, name)))
        d.steady, d.thermal = 1, 0
        d.n_steps, d.n_adj = int(pb.n_steps), int(pb.n_adj)
        d.exec_path = PATH[path]
        d.tol, d.max_steps = float(tol), int(max_steps)
        return d
    if getattr(pb, "periodic", 0) or getattr(pb, "G_x", 0.0) or getattr(pb, "G_y", 0.0):
        raise ValueError("periodic lattices and an external force are not part of the CUDA path")
    for name in ("beta_bar", "q_beta", "kappa_Q", "T_ref"):
        if hasattr(pb, name):
            setattr(d, name, float(getattr(pb, name)))
    d.gb[0], d.gb[1] = float(getattr(pb, "gb_x", 0.0)), float(getattr(pb, "gb_y", 0.0))
    d.heat_x0, d.heat_x1 = int(getattr(pb, "heat_x0", 0)), int(getattr(pb, "heat_x1", -1))
    d.heat_q = float(getattr(pb, "heat_q", 0.0))
    d.kappa_E = float(getattr(pb, "kappa_E", 0.0))
    for name in ("nu", "alpha_bar", "q_alpha", "u_max", "pulse_mean", "pulse_amp", "pulse_period",
                 "rho_out", "K_f", "K_s", "q_K", "kappa_T", "kappa_p"):
        setattr(d, name, float(getattr(pb, name)))
    res = pb.resolved if hasattr(pb, "resolved") else (lambda n: getattr(pb, n))
    d.in_y0, d.in_y1 = int(res("in_y0")), int(res("in_y1"))
    d.out_y0, d.out_y1 = int(res("out_y0")), int(res("out_y1"))
    d.thermal = int(pb.thermal)
    d.steady = int(bool(pb.steady))
    for e in range(4):
        d.t_kind[e] = int(pb.t_kind[e])
        d.t_val[e] = float(pb.t_val[e])
    d.n_steps = int(pb.n_steps)
    d.n_adj = int(pb.n_adj)
    d.checkpoint_every = int(checkpoint_every)
    d.snapshot_type = SNAP[snapshot]
    d.exec_path = PATH[path]
    d.res_steps = int(res_steps)
    d.tol = float(tol)
    d.max_steps = int(max_steps)
    d.warm_start = int(bool(warm_start))
    d.segment_type = SNAP[segment]
    return d


def workspace_size(desc: Desc) -> int:
    L = load()
    n = C.c_size_t(0)
    _check(L.lks_workspace_size(C.byref(desc), C.byref(n)), "lks_workspace_size")
    return int(n.value)


def _check(status: int, what: str, handle=None) -> None:
    if status != 0:
        msg = what
        if handle is not None:
            msg += ": " + load().lks_last_error(handle).decode()
        raise LKSError(status, msg)


def selftest_wait(which: int, device: Optional[torch.device] = None) -> int:
    """Runs one of the library's bounded device waits on a condition that never comes
    true (0: the resident marches' tile flag, 1: the TMA kernels' mbarrier) and
    returns the status the kernel recorded (LKS_ERR_TIMEOUT = 6 when it gave up)."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    scratch = torch.zeros(2, dtype=torch.int32, device=dev)
    rec = C.c_int32(-1)
    with torch.cuda.device(dev):
        stream = torch.cuda.current_stream(dev)
        _check(load().lks_selftest_wait(int(which), C.c_void_p(scratch.data_ptr()), C.c_void_p(stream.cuda_stream),
                                        C.byref(rec)), "lks_selftest_wait")
    return int(rec.value)


def edge_moment_map(A: float, cls: int) -> np.ndarray:
    """Host-only: the 6 x 10 adjoint edge moment map of class ``cls`` (column 9: the
    response to the heat-flux coupling kappa~ T)."""
    out = np.zeros(60)
    _check(load().lks_edge_moment_map(float(A), int(cls),
                                      out.ctypes.data_as(C.POINTER(C.c_double))), "edge map")
    return out.reshape(6, 10)


def edge_objective_map(A: float, cls: int) -> np.ndarray:
    """Host-only: the response of the six flow moments of class ``cls`` to a unit
    boundary objective term in every residual row."""
    out = np.zeros(6)
    _check(load().lks_edge_objective_map(float(A), int(cls),
                                         out.ctypes.data_as(C.POINTER(C.c_double))), "edge objective map")
    return out


class LKS:
    """One problem on one device: owns its workspace (a torch uint8 tensor) and the
    library handle.  Fields are (ny, nx) tensors of the descriptor's real type.

    Every call enqueues its kernels on ``stream`` (torch's current stream when the
    handle was made, unless one is given) and reads its input tensors there.  A
    caller that fills them on another stream orders the two first
    (``h.stream.wait_stream(other)``); a tensor of another dtype, shape or device
    is converted on torch's current stream."""

    def __init__(self, pb, real: str = "f32", checkpoint_every: int = 0, snapshot: str = "f32",
                 device: Optional[torch.device] = None, stream: Optional[torch.cuda.Stream] = None,
                 path: str = "auto", res_steps: int = 0, tol: float = 0.0, max_steps: int = 0,
                 warm_start: bool = False, segment: str = "f32"):
        if not torch.cuda.is_available():
            raise RuntimeError("the LKS library needs a CUDA device")
        self.L = load()
        self.pb = pb
        self.desc = make_desc(pb, real, checkpoint_every, snapshot, path, res_steps, tol, max_steps, warm_start,
                              segment)
        self.dtype = torch.float64 if real == "f64" else torch.float32
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.is3 = hasattr(pb, "nz")
        self.shape = (int(pb.nz), int(pb.ny), int(pb.nx)) if self.is3 else (int(pb.ny), int(pb.nx))
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            nbytes = workspace_size(self.desc)
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            h = C.c_void_p()
            _check(self.L.lks_create(C.byref(self.desc), C.c_void_p(self.workspace.data_ptr()),
                                     C.c_size_t(nbytes), C.c_void_p(self.stream.cuda_stream),
                                     C.byref(h)), "lks_create")
        self.h = h
        self.J = torch.zeros((), dtype=torch.float64, device=self.device)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                self.L.lks_destroy(h)
            except Exception:
                pass
            self.h = None

    # -- helpers ------------------------------------------------------------------------
    def _field(self, t: torch.Tensor) -> torch.Tensor:
        if t.dtype != self.dtype or t.device != self.device or tuple(t.shape) != self.shape:
            t = t.to(device=self.device, dtype=self.dtype).reshape(self.shape)
        return t.contiguous()

    def _ptr(self, t: torch.Tensor):
        return C.c_void_p(t.data_ptr())

    def empty(self) -> torch.Tensor:
        return torch.empty(self.shape, dtype=self.dtype, device=self.device)

    # -- Steps 2-5 ----------------------------------------------------------------------
    def lks_forward(self, gamma: torch.Tensor) -> torch.Tensor:
        g = self._field(gamma)
        _check(self.L.lks_forward(self.h, self._ptr(g), C.c_void_p(self.J.data_ptr())),
               "lks_forward", self.h)
        self._gamma_keep = g
        return self.J

    def alks_adjoint(self) -> None:
        _check(self.L.alks_adjoint(self.h), "alks_adjoint", self.h)

    def lks_sensitivity(self, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        out = self.empty() if out is None else out
        _check(self.L.lks_sensitivity(self.h, self._ptr(out)), "lks_sensitivity", self.h)
        return out

    def gradient(self, gamma: torch.Tensor):
        """(J, dJ/dgamma) with device buffers."""
        J = self.lks_forward(gamma).clone()
        self.alks_adjoint()
        return J, self.lks_sensitivity()

    def gradient_host(self, gamma_host: np.ndarray, grad_host: Optional[np.ndarray] = None):
        """End to end through the C ABI with host buffers (copies inside)."""
        npdt = np.float64 if self.dtype == torch.float64 else np.float32
        g = np.ascontiguousarray(gamma_host, dtype=npdt)
        out = np.empty(self.shape, dtype=npdt) if grad_host is None else grad_host
        J = C.c_double(0.0)
        _check(self.L.lks_gradient_host(self.h, g.ctypes.data_as(C.c_void_p), C.byref(J),
                                        out.ctypes.data_as(C.c_void_p)), "lks_gradient_host", self.h)
        return J.value, out

    # -- state access and single marches ------------------------------------------------
    def set_state(self, gamma, drho, u, v, T=None, t: int = 0) -> None:
        fs = [self._field(x) for x in (gamma, drho, u, v)]
        Tt = self._field(T) if T is not None else fs[1]
        self._keep = fs + [Tt]
        _check(self.L.lks_set_state(self.h, *[self._ptr(x) for x in fs], self._ptr(Tt), int(t)),
               "lks_set_state", self.h)

    def get_state(self):
        out = [self.empty() for _ in range(4)]
        _check(self.L.lks_get_state(self.h, *[self._ptr(x) for x in out]), "lks_get_state", self.h)
        return out  # drho, u, v, T (D3Q19: drho, u, v, w)

    def march(self, n: int) -> None:
        _check(self.L.lks_march(self.h, int(n)), "lks_march", self.h)

    def set_adjoint(self, fields: Sequence[torch.Tensor]) -> None:
        fs = [self._field(f) for f in fields]
        while len(fs) < N_ADJ_FIELDS:
            fs.append(fs[0])
        self._akeep = fs
        arr = (C.c_void_p * N_ADJ_FIELDS)(*[f.data_ptr() for f in fs])
        _check(self.L.alks_set_adjoint(self.h, arr), "alks_set_adjoint", self.h)

    def get_adjoint(self):
        n = N_ADJ_FIELDS_3D if self.is3 else N_ADJ_FIELDS
        out = [self.empty() for _ in range(n)]
        arr = (C.c_void_p * n)(*[f.data_ptr() for f in out])
        _check(self.L.alks_get_adjoint(self.h, arr), "alks_get_adjoint", self.h)
        return out

    def adjoint_march(self, n: int) -> None:
        _check(self.L.alks_march(self.h, int(n)), "alks_march", self.h)

    def query(self) -> Stats:
        s = Stats()
        st = self.L.lks_query(self.h, C.byref(s))
        if st not in (0, s.device_status):
            _check(st, "lks_query", self.h)
        return s


# ---------------------------------------------------------------------------------
# Batched form
# ---------------------------------------------------------------------------------
def batch_options(checkpoint_every: int = 0, snapshot: str = "bf16", tile_config: int = -1,
                  use_graph: bool = True, fwd_column: int = -1, adj_column: int = -1) -> BatchOptions:
    o = BatchOptions()
    o.version = LKS_BATCH_VERSION
    o.checkpoint_every = int(checkpoint_every)
    o.snapshot_type = SNAP[snapshot]
    o.tile_config = int(tile_config)
    o.use_graph = 1 if use_graph else 0
    o.fwd_column = int(fwd_column)
    o.adj_column = int(adj_column)
    return o


def batch_descs(problems) -> "C.Array":
    arr = (Desc * len(problems))()
    for k, pb in enumerate(problems):
        arr[k] = make_desc(pb, "f32")
    return arr


def batch_workspace_size(problems, opt: Optional[BatchOptions] = None) -> int:
    L = load()
    descs = batch_descs(problems)
    n = C.c_size_t(0)
    _check(L.lks_batch_workspace_size(len(problems), descs, C.byref(opt) if opt is not None else None,
                                      C.byref(n)), "lks_batch_workspace_size")
    return int(n.value)


class LKSBatch:
    """Many unsteady FP32 designs of unequal size, marched in lock step by one
    persistent launch per step; a gradient of every design is one call (one CUDA
    graph launch when ``use_graph``)."""

    def __init__(self, problems, checkpoint_every: int = 0, snapshot: str = "bf16", tile_config: int = -1,
                 use_graph: bool = True, device: Optional[torch.device] = None,
                 stream: Optional[torch.cuda.Stream] = None, fwd_column: int = -1, adj_column: int = -1):
        if not torch.cuda.is_available():
            raise RuntimeError("the LKS library needs a CUDA device")
        self.L = load()
        self.problems = list(problems)
        self.n = len(self.problems)
        self.shapes = [(int(p.ny), int(p.nx)) for p in self.problems]
        self.opt = batch_options(checkpoint_every, snapshot, tile_config, use_graph, fwd_column, adj_column)
        self.descs = batch_descs(self.problems)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            n = C.c_size_t(0)
            _check(self.L.lks_batch_workspace_size(self.n, self.descs, C.byref(self.opt), C.byref(n)),
                   "lks_batch_workspace_size")
            self.workspace = torch.empty(int(n.value), dtype=torch.uint8, device=self.device)
            h = C.c_void_p()
            st = self.L.lks_batch_create(self.n, self.descs, C.byref(self.opt),
                                         C.c_void_p(self.workspace.data_ptr()), n,
                                         C.c_void_p(self.stream.cuda_stream), C.byref(h))
            if st != 0:
                raise LKSError(st, "lks_batch_create")
        self.h = h
        self.J = torch.zeros(self.n, dtype=torch.float64, device=self.device)
        self.grads = [torch.empty(s, dtype=torch.float32, device=self.device) for s in self.shapes]
        self._gptr = (C.c_void_p * self.n)()
        self._dptr = (C.c_void_p * self.n)(*[g.data_ptr() for g in self.grads])

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                self.L.lks_batch_destroy(h)
            except Exception:
                pass
            self.h = None

    def gradient(self, gammas: Sequence[torch.Tensor]):
        """(J[n] float64 tensor, [dJ/dgamma per design]) -- the returned tensors are
        reused by the next call."""
        if len(gammas) != self.n:
            raise ValueError("one gamma per design")
        keep = []
        for k, (g, s) in enumerate(zip(gammas, self.shapes)):
            if g.dtype != torch.float32 or g.device != self.device or tuple(g.shape) != s or not g.is_contiguous():
                g = g.to(device=self.device, dtype=torch.float32).reshape(s).contiguous()
            keep.append(g)
            self._gptr[k] = g.data_ptr()
        st = self.L.lks_batch_gradient(self.h, self._gptr, C.c_void_p(self.J.data_ptr()), self._dptr)
        if st != 0:
            raise LKSError(st, "lks_batch_gradient: " + self.L.lks_batch_last_error(self.h).decode())
        self._keep = keep  # inputs stay alive until the stream has consumed them
        return self.J, self.grads

    def query(self) -> BatchStats:
        s = BatchStats()
        _check(self.L.lks_batch_query(self.h, C.byref(s)), "lks_batch_query")
        return s
