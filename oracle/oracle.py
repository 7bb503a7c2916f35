"""ctypes front end of the FP64 CPU oracle (``lks_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  Nothing in the product package may import
this module.

Every function here only marshals arrays into the C oracle and strings its steps
together in the order of the paper's procedure (Sec. 2.7, Steps 2-5):
state by LKS, objective, adjoint by ALKS, sensitivity.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lks_oracle.c")
_SRC3 = os.path.join(_HERE, "lks3d_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liblks_oracle.so")
_lock = threading.Lock()
_lib = None

NADJ = 9
ADJ_NAMES = ("rho_t", "ux_t", "uy_t", "sxx_t", "sxy_t", "syy_t", "T_t", "qx_t", "qy_t")


class OrcProblem(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("nu", C.c_double),
        ("alpha_bar", C.c_double), ("q_alpha", C.c_double),
        ("u_max", C.c_double),
        ("pulse_mean", C.c_double), ("pulse_amp", C.c_double), ("pulse_period", C.c_double),
        ("in_y0", C.c_int), ("in_y1", C.c_int),
        ("out_y0", C.c_int), ("out_y1", C.c_int),
        ("rho_out", C.c_double),
        ("thermal", C.c_int),
        ("K_f", C.c_double), ("K_s", C.c_double), ("q_K", C.c_double),
        ("t_kind", C.c_int * 4),
        ("t_val", C.c_double * 4),
        ("kappa_T", C.c_double),
        ("kappa_p", C.c_double),
        ("periodic", C.c_int),
        ("G_x", C.c_double), ("G_y", C.c_double),
        ("beta_bar", C.c_double), ("q_beta", C.c_double), ("kappa_Q", C.c_double),
        ("gb_x", C.c_double), ("gb_y", C.c_double), ("T_ref", C.c_double),
        ("heat_x0", C.c_int), ("heat_x1", C.c_int), ("heat_q", C.c_double),
        ("kappa_E", C.c_double),
    ]


class OrcProblem3(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("nu", C.c_double),
        ("alpha_bar", C.c_double), ("q_alpha", C.c_double),
        ("u_max", C.c_double),
        ("rho_out", C.c_double),
        ("profile", C.c_int),
        ("kappa_p", C.c_double),
    ]


NADJ3 = 10
ADJ3_NAMES = ("rho_t", "ux_t", "uy_t", "uz_t", "sxx_t", "sxy_t", "sxz_t", "syy_t", "syz_t", "szz_t")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, OpenMP).  Returns the library path."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
                os.path.getmtime(_SRC), os.path.getmtime(_SRC3)):
            return _LIB
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, _SRC3, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.POINTER(C.c_double)
        PP = C.POINTER(P)
        prob = C.POINTER(OrcProblem)
        L.orc_forward_node.argtypes = [prob, P, C.c_double, P, P, P, P, C.c_int, C.c_int, P]
        L.orc_forward_step.argtypes = [prob, P, C.c_double, P, P, P, P, P, P, P, P]
        L.orc_objective.argtypes = [prob, P, P, P, P]
        L.orc_objective.restype = C.c_double
        L.orc_dJdu_node.argtypes = [prob, P, P, P, C.c_int, C.c_int, P, P]
        L.orc_bc_flow.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                  C.POINTER(C.c_int), P, P, C.c_double, P]
        L.orc_pressure_drop.argtypes = [prob, P]
        L.orc_pressure_drop.restype = C.c_double
        L.orc_energy_loss.argtypes = [prob, P, P, P]
        L.orc_energy_loss.restype = C.c_double
        L.orc_objective_total.argtypes = [prob, P, P, P, P, P]
        L.orc_objective_total.restype = C.c_double
        L.orc_bc_thermal.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                     C.POINTER(C.c_int), P, P]
        L.orc_adjoint_step.argtypes = [prob, P, P, P, P, P, P, PP, PP, P]
        L.orc_adjoint_eq.argtypes = [prob, P, P, P, PP, P, P, P, P, P]
        L.orc_adjoint_node.argtypes = [prob, P, P, P, P, P, P, P, P, C.c_int, C.c_int, P]
        L.orc_sensitivity_accum.argtypes = [prob, P, P, P, P, PP, P]
        L.orc_forward.argtypes = [prob, P, C.c_int, C.c_int, P, P, P, P, P, P]
        L.orc_forward.restype = C.c_double
        L.orc_steady_adjoint.argtypes = [prob, P, P, P, P, C.c_int, P, P]
        L.orc_steady_adjoint.restype = C.c_double
        L.orc_unsteady_adjoint.argtypes = [prob, P, C.c_int, P, P, P]
        p3 = C.POINTER(OrcProblem3)
        IP = C.POINTER(C.c_int)
        L.orc3_lattice.argtypes = [IP, P]
        L.orc3_feq_moments.argtypes = [C.c_double, C.c_double, P, P, P]
        L.orc3_forward_node.argtypes = [p3, P, P, PP, C.c_int, C.c_int, C.c_int, P]
        L.orc3_forward_step.argtypes = [p3, P, P, P, P, P, P, P, P, P]
        L.orc3_objective.argtypes = [p3, P, P, P, P]
        L.orc3_objective.restype = C.c_double
        L.orc3_dJdu_node.argtypes = [p3, P, PP, C.c_int, C.c_int, C.c_int, P]
        L.orc3_bc_flow.argtypes = [IP, C.c_int, C.c_double, IP, P, P, C.c_double]
        L.orc3_pressure_drop.argtypes = [p3, P]
        L.orc3_pressure_drop.restype = C.c_double
        L.orc3_objective_total.argtypes = [p3, P, P, P, P, P]
        L.orc3_objective_total.restype = C.c_double
        L.orc3_adjoint_eq.argtypes = [p3, PP, PP, PP]
        L.orc3_adjoint_node.argtypes = [p3, P, PP, PP, C.c_int, C.c_int, C.c_int, P]
        L.orc3_adjoint_step.argtypes = [p3, P, PP, PP, PP, PP, P]
        L.orc3_sensitivity_accum.argtypes = [p3, P, PP, PP, P]
        L.orc3_forward.argtypes = [p3, P, C.c_int, P, P, P, P, P, P]
        L.orc3_forward.restype = C.c_double
        L.orc3_steady_adjoint.argtypes = [p3, P, P, P, P, C.c_int, P, P]
        L.orc3_steady_adjoint.restype = C.c_double
        L.orc3_unsteady_adjoint.argtypes = [p3, P, C.c_int, P, P, P]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_get_threads.restype = C.c_int
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _pp(arrs):
    P = C.POINTER(C.c_double)
    return (P * len(arrs))(*[_p(a) for a in arrs])


def make_problem(pb) -> OrcProblem:
    """OrcProblem from an ``inputs.Problem`` (or any object with the same fields)."""
    s = OrcProblem()
    for name, _ in OrcProblem._fields_:
        if name in ("t_kind", "t_val"):
            continue
        if not hasattr(pb, name) and name in ("periodic", "G_x", "G_y", "beta_bar", "q_beta", "kappa_Q", "gb_x",
                                              "gb_y", "T_ref", "heat_x0", "heat_q", "kappa_E"):
            continue  # fields a problem description may leave out: zero
        if not hasattr(pb, name) and name == "heat_x1":
            s.heat_x1 = -1  # no heated segment
            continue
        val = pb.resolved(name) if hasattr(pb, "resolved") else getattr(pb, name)
        setattr(s, name, type(getattr(s, name))(val))
    for e in range(4):
        s.t_kind[e] = int(pb.t_kind[e])
        s.t_val[e] = float(pb.t_val[e])
    return s


class State:
    """rho, u, v, T fields, each (ny, nx) float64."""

    def __init__(self, ny: int, nx: int):
        self.rho = np.ones((ny, nx))
        self.u = np.zeros((ny, nx))
        self.v = np.zeros((ny, nx))
        self.T = np.zeros((ny, nx))

    def copy(self) -> "State":
        s = State(*self.rho.shape)
        s.rho, s.u, s.v, s.T = self.rho.copy(), self.u.copy(), self.v.copy(), self.T.copy()
        return s


def _g(gamma):
    return np.ascontiguousarray(gamma, dtype=np.float64)


def forward(pb, gamma: np.ndarray, n_steps: int, state: Optional[State] = None, t0: int = 0,
            traj: bool = False, accumulate_J: bool = False):
    """LKS march (Step 2).  Returns (state, residual, traj or None, J_sum)."""
    L = lib()
    prob = make_problem(pb)
    g = _g(gamma)
    st = state.copy() if state is not None else State(pb.ny, pb.nx)
    tr = np.zeros((n_steps + 1, 3, pb.ny, pb.nx)) if traj else None
    Jacc = C.c_double(0.0)
    res = L.orc_forward(C.byref(prob), _p(g), int(t0), int(n_steps), _p(st.rho), _p(st.u),
                        _p(st.v), _p(st.T), _p(tr) if traj else None,
                        C.byref(Jacc) if accumulate_J else None)
    return st, res, tr, Jacc.value


def forward_to_steady(pb, gamma, tol=1e-13, max_steps=200000, chunk=500, state=None):
    """LKS march until max |u(t) - u(t-1)| < tol (or max_steps)."""
    st = state
    done = 0
    res = np.inf
    while done < max_steps:
        st, res, _, _ = forward(pb, gamma, chunk, state=st)
        done += chunk
        if res < tol:
            break
    return st, res, done


def forward_step(pb, gamma, t, st: State) -> State:
    L = lib()
    prob = make_problem(pb)
    g = _g(gamma)
    out = State(pb.ny, pb.nx)
    L.orc_forward_step(C.byref(prob), _p(g), float(t), _p(st.rho), _p(st.u), _p(st.v), _p(st.T),
                       _p(out.rho), _p(out.u), _p(out.v), _p(out.T))
    return out


def forward_node(pb, gamma, t, st: State, i: int, j: int) -> np.ndarray:
    L = lib()
    prob = make_problem(pb)
    g = _g(gamma)
    o = np.zeros(4)
    L.orc_forward_node(C.byref(prob), _p(g), float(t), _p(st.rho), _p(st.u), _p(st.v), _p(st.T),
                       int(i), int(j), _p(o))
    return o


def objective(pb, gamma, st: State) -> float:
    """J = J_O + kappa_p J_p + kappa_E J_E of one state (Step 3)."""
    L = lib()
    prob = make_problem(pb)
    return float(L.orc_objective_total(C.byref(prob), _p(_g(gamma)), _p(st.rho), _p(st.u), _p(st.v),
                                       _p(st.T)))


def pressure_drop(pb, st: State) -> float:
    """J_p = sum_in p - sum_out p with p = rho / 3 (unweighted)."""
    return float(lib().orc_pressure_drop(C.byref(make_problem(pb)), _p(st.rho)))


def energy_loss(pb, st: State) -> float:
    """J_E = sum over inlet and outlet nodes of -n.u (p + |u|^2 / 2) (unweighted)."""
    return float(lib().orc_energy_loss(C.byref(make_problem(pb)), _p(st.rho), _p(st.u), _p(st.v)))


def dJdu(pb, gamma, st: State):
    """dJ_O/du, dJ_O/dv at every node."""
    L = lib()
    prob = make_problem(pb)
    g = _g(gamma)
    ju = np.zeros((pb.ny, pb.nx))
    jv = np.zeros((pb.ny, pb.nx))
    a, b = C.c_double(), C.c_double()
    for j in range(pb.ny):
        for i in range(pb.nx):
            L.orc_dJdu_node(C.byref(prob), _p(g), _p(st.u), _p(st.v), i, j, C.byref(a), C.byref(b))
            ju[j, i], jv[j, i] = a.value, b.value
    return ju, jv


def adjoint_step(pb, gamma, st1: State, st0: State, adj1: np.ndarray) -> np.ndarray:
    """One ALKS step: adjoint (NADJ, ny, nx) at level t+1 -> level t."""
    L = lib()
    prob = make_problem(pb)
    a1 = np.ascontiguousarray(adj1, dtype=np.float64)
    a0 = np.zeros_like(a1)
    work = np.zeros((5, pb.ny, pb.nx))
    L.orc_adjoint_step(C.byref(prob), _p(_g(gamma)), _p(st1.u), _p(st1.v), _p(st0.u), _p(st0.v),
                       _p(st0.T), _pp([a1[q] for q in range(NADJ)]),
                       _pp([a0[q] for q in range(NADJ)]), _p(work))
    return a0


def adjoint_eq(pb, gamma, st: State, adj: np.ndarray) -> np.ndarray:
    """Adjoint equilibrium coefficients (P, Vx, Vy, G) at every node, Eqs. (afeq), (ageq)."""
    L = lib()
    prob = make_problem(pb)
    a = np.ascontiguousarray(adj, dtype=np.float64)
    out = np.zeros((5, pb.ny, pb.nx))
    L.orc_adjoint_eq(C.byref(prob), _p(_g(gamma)), _p(st.u), _p(st.v),
                     _pp([a[q] for q in range(NADJ)]), _p(out[0]), _p(out[1]), _p(out[2]),
                     _p(out[3]), _p(out[4]))
    return out[:4].copy()


def adjoint_gather(pb, gamma, PVG: np.ndarray, st0: State) -> np.ndarray:
    """Adjoint moments at level t from given equilibrium coefficients (P, Vx, Vy, G)
    of level t+1 (gather, boundary rule, sources, moments) at every node."""
    L = lib()
    prob = make_problem(pb)
    g = _g(gamma)
    c = [np.ascontiguousarray(PVG[q], dtype=np.float64) for q in range(4)]
    out = np.zeros((NADJ, pb.ny, pb.nx))
    o = np.zeros(NADJ)
    for j in range(pb.ny):
        for i in range(pb.nx):
            L.orc_adjoint_node(C.byref(prob), _p(g), _p(c[0]), _p(c[1]), _p(c[2]), _p(c[3]),
                               _p(st0.u), _p(st0.v), _p(st0.T), i, j, _p(o))
            out[:, j, i] = o
    return out


def sensitivity_level(pb, gamma, st: State, adj: np.ndarray) -> np.ndarray:
    """Sensitivity integrand of one level (interior nodes, zero on edges)."""
    L = lib()
    prob = make_problem(pb)
    a = np.ascontiguousarray(adj, dtype=np.float64)
    s = np.zeros((pb.ny, pb.nx))
    L.orc_sensitivity_accum(C.byref(prob), _p(_g(gamma)), _p(st.u), _p(st.v), _p(st.T),
                            _pp([a[q] for q in range(NADJ)]), _p(s))
    return s


def steady_adjoint(pb, gamma, st: State, n_iter: int):
    """ALKS iterated with the frozen state (Step 4) and the sensitivity (Step 5).
    Returns (adjoint (NADJ, ny, nx), dJ/dgamma (ny, nx), last change)."""
    L = lib()
    prob = make_problem(pb)
    adj = np.zeros((NADJ, pb.ny, pb.nx))
    sens = np.zeros((pb.ny, pb.nx))
    res = L.orc_steady_adjoint(C.byref(prob), _p(_g(gamma)), _p(st.u), _p(st.v), _p(st.T),
                               int(n_iter), _p(adj), _p(sens))
    return adj, sens, res


def unsteady_adjoint(pb, gamma, traj: np.ndarray):
    """ALKS marched backward over a stored trajectory (levels 0..n)."""
    L = lib()
    prob = make_problem(pb)
    n = traj.shape[0] - 1
    tr = np.ascontiguousarray(traj, dtype=np.float64)
    adj = np.zeros((NADJ, pb.ny, pb.nx))
    sens = np.zeros((pb.ny, pb.nx))
    L.orc_unsteady_adjoint(C.byref(prob), _p(_g(gamma)), int(n), _p(tr), _p(adj), _p(sens))
    return adj, sens


def steady_gradient(pb, gamma, n_steps: Optional[int] = None, n_adj: Optional[int] = None):
    """Steps 2-5 for a steady problem with fixed step counts.
    Returns dict(J, dJdgamma, state, adjoint)."""
    n_steps = pb.n_steps if n_steps is None else n_steps
    n_adj = pb.n_adj if n_adj is None else n_adj
    st, _, _, _ = forward(pb, gamma, n_steps)
    J = objective(pb, gamma, st)
    adj, sens, _ = steady_adjoint(pb, gamma, st, n_adj)
    return dict(J=J, dJdgamma=sens, state=st, adjoint=adj)


def unsteady_gradient(pb, gamma, n_steps: Optional[int] = None):
    """Steps 2-5 for an unsteady problem; J = sum over levels 1..n of J_O."""
    n_steps = pb.n_steps if n_steps is None else n_steps
    st, _, tr, J = forward(pb, gamma, n_steps, traj=True, accumulate_J=True)
    adj, sens = unsteady_adjoint(pb, gamma, tr)
    return dict(J=J, dJdgamma=sens, state=st, adjoint=adj, traj=tr)


def bc_flow(n, pressure: bool, A: float, known: np.ndarray, unknown_mask, kT: float = 0.0, jb: float = 0.0,
            jbv=None):
    """Least-squares adjoint boundary rule for one node (flow lattice); jb is the
    boundary objective term added to every row, jbv (9 values, optional) a term per
    row."""
    L = lib()
    f = np.ascontiguousarray(known, dtype=np.float64).copy()
    um = (C.c_int * 9)(*[int(x) for x in unknown_mask])
    mult = np.zeros(2)
    jv = None if jbv is None else np.ascontiguousarray(jbv, dtype=np.float64)
    L.orc_bc_flow(int(n[0]), int(n[1]), int(pressure), float(A), float(kT), um, _p(f), _p(mult), float(jb),
                  None if jv is None else _p(jv))
    return f, mult


def bc_thermal(n, flux: bool, B: float, un: float, known: np.ndarray, unknown_mask):
    """Least-squares adjoint boundary rule for one node (thermal lattice)."""
    L = lib()
    g = np.ascontiguousarray(known, dtype=np.float64).copy()
    um = (C.c_int * 9)(*[int(x) for x in unknown_mask])
    mult = np.zeros(1)
    L.orc_bc_thermal(int(n[0]), int(n[1]), int(flux), float(B), float(un), um, _p(g), _p(mult))
    return g, float(mult[0])


# ---------------------------------------------------------------------------------
# Three dimensions (D3Q19, steady duct; ``lks3d_oracle.c``)
# ---------------------------------------------------------------------------------
def make_problem3(pb) -> OrcProblem3:
    s = OrcProblem3()
    for name, _ in OrcProblem3._fields_:
        setattr(s, name, type(getattr(s, name))(getattr(pb, name)))
    return s


class State3:
    """rho, u, v, w fields, each (nz, ny, nx) float64."""

    def __init__(self, nz: int, ny: int, nx: int):
        self.rho = np.ones((nz, ny, nx))
        self.u = np.zeros((nz, ny, nx))
        self.v = np.zeros((nz, ny, nx))
        self.w = np.zeros((nz, ny, nx))

    def copy(self) -> "State3":
        s = State3(*self.rho.shape)
        s.rho, s.u, s.v, s.w = self.rho.copy(), self.u.copy(), self.v.copy(), self.w.copy()
        return s

    def vel(self):
        return [self.u, self.v, self.w]


def lattice3():
    """(c (19, 3) int, w (19,)) of the 3-D oracle."""
    c = (C.c_int * 57)()
    w = np.zeros(19)
    lib().orc3_lattice(c, _p(w))
    return np.array(list(c), dtype=int).reshape(19, 3), w


def feq_moments3(A: float, rho: float, u, grad) -> np.ndarray:
    out = np.zeros(10)
    lib().orc3_feq_moments(float(A), float(rho), _p(np.asarray(u, dtype=np.float64).copy()),
                           _p(np.ascontiguousarray(grad, dtype=np.float64).reshape(9).copy()), _p(out))
    return out


def forward3(pb, gamma, n_steps: int, state: Optional[State3] = None, traj: bool = False,
             accumulate_J: bool = False):
    """3-D LKS march.  Returns (state, residual, traj or None, J_sum)."""
    L = lib()
    prob = make_problem3(pb)
    st = state.copy() if state is not None else State3(pb.nz, pb.ny, pb.nx)
    tr = np.zeros((n_steps + 1, 3, pb.nz, pb.ny, pb.nx)) if traj else None
    Jacc = C.c_double(0.0)
    res = L.orc3_forward(C.byref(prob), _p(_g(gamma)), int(n_steps), _p(st.rho), _p(st.u), _p(st.v),
                         _p(st.w), _p(tr) if traj else None, C.byref(Jacc) if accumulate_J else None)
    return st, res, tr, Jacc.value


def forward_step3(pb, gamma, st: State3) -> State3:
    out = State3(pb.nz, pb.ny, pb.nx)
    lib().orc3_forward_step(C.byref(make_problem3(pb)), _p(_g(gamma)), _p(st.rho), _p(st.u), _p(st.v),
                            _p(st.w), _p(out.rho), _p(out.u), _p(out.v), _p(out.w))
    return out


def objective3(pb, gamma, st: State3) -> float:
    """J = J_O + kappa_p J_p of one state."""
    return float(lib().orc3_objective_total(C.byref(make_problem3(pb)), _p(_g(gamma)), _p(st.rho), _p(st.u),
                                            _p(st.v), _p(st.w)))


def dissipation3(pb, gamma, st: State3) -> float:
    """J_O alone (total dissipation)."""
    return float(lib().orc3_objective(C.byref(make_problem3(pb)), _p(_g(gamma)), _p(st.u), _p(st.v),
                                      _p(st.w)))


def pressure_drop3(pb, st: State3) -> float:
    """J_p = sum_in p - sum_out p with p = rho / 3 (unweighted)."""
    return float(lib().orc3_pressure_drop(C.byref(make_problem3(pb)), _p(st.rho)))


def dJdu3(pb, gamma, st: State3) -> np.ndarray:
    L = lib()
    prob = make_problem3(pb)
    g = _g(gamma)
    out = np.zeros((3, pb.nz, pb.ny, pb.nx))
    o = np.zeros(3)
    for k in range(pb.nz):
        for j in range(pb.ny):
            for i in range(pb.nx):
                L.orc3_dJdu_node(C.byref(prob), _p(g), _pp(st.vel()), i, j, k, _p(o))
                out[:, k, j, i] = o
    return out


def adjoint_eq3(pb, st: State3, adj: np.ndarray) -> np.ndarray:
    """(P, Vx, Vy, Vz) at every node from the adjoint fields and the state."""
    a = np.ascontiguousarray(adj, dtype=np.float64)
    out = np.zeros((4, pb.nz, pb.ny, pb.nx))
    lib().orc3_adjoint_eq(C.byref(make_problem3(pb)), _pp(st.vel()), _pp([a[q] for q in range(NADJ3)]),
                          _pp([out[q] for q in range(4)]))
    return out


def adjoint_gather3(pb, gamma, PV: np.ndarray, st0: State3) -> np.ndarray:
    """Adjoint moments at level t from the coefficients PV of level t+1."""
    L = lib()
    prob = make_problem3(pb)
    g = _g(gamma)
    c = [np.ascontiguousarray(PV[q], dtype=np.float64) for q in range(4)]
    out = np.zeros((NADJ3, pb.nz, pb.ny, pb.nx))
    o = np.zeros(NADJ3)
    for k in range(pb.nz):
        for j in range(pb.ny):
            for i in range(pb.nx):
                L.orc3_adjoint_node(C.byref(prob), _p(g), _pp(c), _pp(st0.vel()), i, j, k, _p(o))
                out[:, k, j, i] = o
    return out


def adjoint_step3(pb, gamma, st1: State3, st0: State3, adj1: np.ndarray) -> np.ndarray:
    a1 = np.ascontiguousarray(adj1, dtype=np.float64)
    a0 = np.zeros_like(a1)
    work = np.zeros((4, pb.nz, pb.ny, pb.nx))
    lib().orc3_adjoint_step(C.byref(make_problem3(pb)), _p(_g(gamma)), _pp(st1.vel()), _pp(st0.vel()),
                            _pp([a1[q] for q in range(NADJ3)]), _pp([a0[q] for q in range(NADJ3)]), _p(work))
    return a0


def steady_adjoint3(pb, gamma, st: State3, n_iter: int):
    adj = np.zeros((NADJ3, pb.nz, pb.ny, pb.nx))
    sens = np.zeros((pb.nz, pb.ny, pb.nx))
    res = lib().orc3_steady_adjoint(C.byref(make_problem3(pb)), _p(_g(gamma)), _p(st.u), _p(st.v),
                                    _p(st.w), int(n_iter), _p(adj), _p(sens))
    return adj, sens, res


def unsteady_adjoint3(pb, gamma, traj: np.ndarray):
    n = traj.shape[0] - 1
    tr = np.ascontiguousarray(traj, dtype=np.float64)
    adj = np.zeros((NADJ3, pb.nz, pb.ny, pb.nx))
    sens = np.zeros((pb.nz, pb.ny, pb.nx))
    lib().orc3_unsteady_adjoint(C.byref(make_problem3(pb)), _p(_g(gamma)), int(n), _p(tr), _p(adj), _p(sens))
    return adj, sens


def steady_gradient3(pb, gamma, n_steps: Optional[int] = None, n_adj: Optional[int] = None):
    """Steps 2-5 for a steady 3-D problem with fixed step counts."""
    n_steps = pb.n_steps if n_steps is None else n_steps
    n_adj = pb.n_adj if n_adj is None else n_adj
    st, _, _, _ = forward3(pb, gamma, n_steps)
    J = objective3(pb, gamma, st)
    adj, sens, _ = steady_adjoint3(pb, gamma, st, n_adj)
    return dict(J=J, dJdgamma=sens, state=st, adjoint=adj)


def bc_flow3(n, pressure: bool, A: float, known: np.ndarray, unknown_mask, jb: float = 0.0):
    f = np.ascontiguousarray(known, dtype=np.float64).copy()
    nn = (C.c_int * 3)(*[int(x) for x in n])
    um = (C.c_int * 19)(*[int(x) for x in unknown_mask])
    mult = np.zeros(3)
    lib().orc3_bc_flow(nn, int(pressure), float(A), um, _p(f), _p(mult), float(jb))
    return f, mult


def forward_node3(pb, gamma, st: State3, i: int, j: int, k: int) -> np.ndarray:
    """(rho, u, v, w) at one node after one step from the state st."""
    o = np.zeros(4)
    lib().orc3_forward_node(C.byref(make_problem3(pb)), _p(_g(gamma)), _p(st.rho), _pp(st.vel()), int(i),
                            int(j), int(k), _p(o))
    return o


def adjoint_node3(pb, gamma, PV: np.ndarray, st0: State3, i: int, j: int, k: int) -> np.ndarray:
    """Adjoint moments at one node from the coefficients PV of the previous level."""
    o = np.zeros(NADJ3)
    c = [np.ascontiguousarray(PV[q], dtype=np.float64) for q in range(4)]
    lib().orc3_adjoint_node(C.byref(make_problem3(pb)), _p(_g(gamma)), _pp(c), _pp(st0.vel()), int(i), int(j),
                            int(k), _p(o))
    return o
