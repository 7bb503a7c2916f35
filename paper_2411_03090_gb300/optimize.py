"""The optimisation loop of Sec. 2.7 (Steps 1-7) around the gamma -> J function.

Step 1   the design field gamma is initialised on the design domain;
Steps 2-3 state by LKS and the objective J (``LKSObjective`` forward, i.e.
         ``lks_forward``), and the constraint G;
Steps 4-5 adjoint by ALKS and the sensitivities J', G' (``LKSObjective`` backward,
         i.e. ``alks_adjoint`` + ``lks_sensitivity``, chained through the filter and
         the projection by torch autograd);
Step 6   gamma is updated by the method of moving asymptotes (MMA);
Step 7   repeat until the design stops changing or the iteration limit is reached.

The constraint is the flow-path area (Eq. constraint_pipebend):
G = sum_D gamma_phys / |D| - V_max <= 0 over the design domain D.  The design
variables pass through a density filter with a linear (cone) kernel of radius R and
the Heaviside projection of Wang, Lazarov and Sigmund (2011) with threshold eta and
steepness beta, which the paper applies with R = 2.4 dx and beta doubled every 100
iterations (heat-sink example).  Nodes outside D keep gamma = 1 (fluid).

MMA follows Svanberg's published method (1987) for one constraint: moving
asymptotes L, U adapted by the sign of the last two steps, convex separable
approximations with the p, q coefficients, move limits, and the subproblem solved
through its one-dimensional dual by bisection on the multiplier.

Everything runs on the caller's device with torch element-wise operations; the
flow and adjoint marches are the CUDA library's.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import torch


# ------------------------------------------------------------------------------------
# Filter and projection
# ------------------------------------------------------------------------------------
def cone_kernel(R: float, dtype=torch.float64, device=None) -> torch.Tensor:
    """Weights max(0, R - |d|) on the integer offsets |d| < R, as a 1 x 1 x k x k
    convolution kernel (unnormalised)."""
    r = int(math.ceil(R)) - (1 if float(R).is_integer() else 0)
    ax = torch.arange(-r, r + 1, dtype=dtype, device=device)
    d = torch.sqrt(ax[:, None] ** 2 + ax[None, :] ** 2)
    w = torch.clamp(R - d, min=0.0)
    return w[None, None]


def density_filter(x: torch.Tensor, R: float) -> torch.Tensor:
    """Cone-weighted average of a 2-D field over the radius R, normalised at every
    node by the weights that fall inside the field (no padding bias at edges)."""
    if R <= 1.0:
        return x
    k = cone_kernel(R, x.dtype, x.device)
    pad = k.shape[-1] // 2
    num = torch.nn.functional.conv2d(x[None, None], k, padding=pad)[0, 0]
    den = torch.nn.functional.conv2d(torch.ones_like(x)[None, None], k, padding=pad)[0, 0]
    return num / den


def heaviside_projection(x: torch.Tensor, beta: float, eta: float = 0.5) -> torch.Tensor:
    """Smoothed Heaviside projection: (tanh(beta eta) + tanh(beta (x - eta))) /
    (tanh(beta eta) + tanh(beta (1 - eta))); maps 0 -> 0 and 1 -> 1, and tends to a
    step at eta as beta grows."""
    a = math.tanh(beta * eta)
    return (a + torch.tanh(beta * (x - eta))) / (a + math.tanh(beta * (1.0 - eta)))


# ------------------------------------------------------------------------------------
# MMA (Svanberg 1987), one constraint
# ------------------------------------------------------------------------------------
@dataclass
class MMAState:
    """Iterates and asymptotes carried between MMA steps."""

    xold1: Optional[torch.Tensor] = None
    xold2: Optional[torch.Tensor] = None
    low: Optional[torch.Tensor] = None
    upp: Optional[torch.Tensor] = None
    iteration: int = 0


def mma_update(x: torch.Tensor, df0: torch.Tensor, f1: float, df1: torch.Tensor, st: MMAState,
               xmin: float = 0.0, xmax: float = 1.0, move: float = 0.2, asyinit: float = 0.5,
               asydec: float = 0.7, asyinc: float = 1.2, raa0: float = 1e-5, asymin: float = 0.01) -> torch.Tensor:
    """One MMA step for  min f0(x)  s.t.  f1(x) <= 0,  xmin <= x <= xmax.

    x, df0, df1: the design variables and the gradients of f0 and f1 (same shape);
    f1: the constraint value at x.  Returns the new x and updates st in place.
    The asymptotes stay between asymin and 10 times the variable range from x; with
    asymin = 0.01 the iterates settle to about that fraction of the range, which a
    smaller asymin refines."""
    span = xmax - xmin
    st.iteration += 1
    if st.iteration <= 2 or st.low is None:
        low = x - asyinit * span
        upp = x + asyinit * span
    else:
        sgn = (x - st.xold1) * (st.xold1 - st.xold2)
        fac = torch.where(sgn > 0, torch.full_like(x, asyinc),
                          torch.where(sgn < 0, torch.full_like(x, asydec), torch.ones_like(x)))
        low = x - fac * (st.xold1 - st.low)
        upp = x + fac * (st.upp - st.xold1)
        low = torch.minimum(torch.maximum(low, x - 10.0 * span), x - asymin * span)
        upp = torch.maximum(torch.minimum(upp, x + 10.0 * span), x + asymin * span)
    alpha = torch.maximum(torch.maximum(low + 0.1 * (x - low), x - move * span), torch.full_like(x, xmin))
    beta = torch.minimum(torch.minimum(upp - 0.1 * (upp - x), x + move * span), torch.full_like(x, xmax))

    ux2 = (upp - x) ** 2
    xl2 = (x - low) ** 2
    reg = raa0 / span
    p0 = ux2 * (torch.clamp(df0, min=0.0) + 0.001 * df0.abs() + reg)
    q0 = xl2 * (torch.clamp(-df0, min=0.0) + 0.001 * df0.abs() + reg)
    p1 = ux2 * torch.clamp(df1, min=0.0)
    q1 = xl2 * torch.clamp(-df1, min=0.0)
    r1 = f1 - float((p1 / (upp - x) + q1 / (x - low)).sum())

    def x_of(lam: float) -> torch.Tensor:
        P = torch.sqrt(p0 + lam * p1)
        Q = torch.sqrt(q0 + lam * q1)
        xs = (P * low + Q * upp) / (P + Q)
        return torch.minimum(torch.maximum(xs, alpha), beta)

    def g_of(xs: torch.Tensor) -> float:
        return float((p1 / (upp - xs) + q1 / (xs - low)).sum()) + r1

    xn = x_of(0.0)
    if g_of(xn) > 0.0:  # the constraint binds: the dual maximum has lam > 0
        lo, hi = 0.0, 1.0
        while g_of(x_of(hi)) > 0.0 and hi < 1e30:
            hi *= 10.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if g_of(x_of(mid)) > 0.0:
                lo = mid
            else:
                hi = mid
            if hi - lo <= 1e-12 * max(1.0, hi):
                break
        xn = x_of(hi)
    st.xold2 = st.xold1
    st.xold1 = x.clone()
    st.low, st.upp = low, upp
    return xn


# ------------------------------------------------------------------------------------
# The loop
# ------------------------------------------------------------------------------------
@dataclass
class History:
    J: List[float] = field(default_factory=list)
    G: List[float] = field(default_factory=list)
    change: List[float] = field(default_factory=list)
    beta: List[float] = field(default_factory=list)


def physical_field(xd: torch.Tensor, mask: torch.Tensor, R: float, beta: float, eta: float = 0.5) -> torch.Tensor:
    """gamma on the whole lattice from the design variables xd (same shape as the
    lattice; only the entries inside the design mask are used): filtered, projected
    inside D, 1 outside."""
    full = torch.where(mask, xd, torch.ones_like(xd))
    phys = heaviside_projection(density_filter(full, R), beta, eta)
    return torch.where(mask, phys, torch.ones_like(xd))


def optimize(objective_fn: Callable[[torch.Tensor], torch.Tensor], mask: torch.Tensor, vmax: float,
             n_iter: int = 50, x0: Optional[torch.Tensor] = None, R: float = 2.4, beta0: float = 1.0,
             beta_every: int = 100, beta_max: float = 64.0, eta: float = 0.5, move: float = 0.2,
             tol_change: float = 1e-3, callback=None):
    """Steps 1-7 of Sec. 2.7.

    objective_fn: gamma (whole lattice, float64 tensor with requires_grad) -> J, a
    scalar tensor whose backward gives dJ/dgamma (e.g. ``LKSObjective`` of an LKS
    handle).  mask: boolean design domain D.  vmax: the area fraction bound of
    Eq. (constraint_pipebend).  Returns (gamma_phys, design variables, History).
    The loop stops after n_iter iterations, or earlier when the largest change of a
    design variable falls below tol_change (at the final beta)."""
    dev = mask.device
    nd = int(mask.sum())
    x = (torch.full(mask.shape, vmax, dtype=torch.float64, device=dev) if x0 is None
         else x0.to(dev, torch.float64).clone())
    st = MMAState()
    hist = History()
    beta = beta0
    for it in range(n_iter):
        xv = x.detach().requires_grad_(True)
        phys = physical_field(xv, mask, R, beta, eta)
        J = objective_fn(phys)
        G = torch.where(mask, phys, torch.zeros_like(phys)).sum() / nd - vmax
        dJ, = torch.autograd.grad(J, xv, retain_graph=True)
        dG, = torch.autograd.grad(G, xv)
        d = mask
        xn_d = mma_update(x[d], dJ[d].to(torch.float64), float(G.detach()), dG[d].to(torch.float64), st, move=move)
        change = float((xn_d - x[d]).abs().max())
        x = x.clone()
        x[d] = xn_d
        hist.J.append(float(J.detach()))
        hist.G.append(float(G.detach()))
        hist.change.append(change)
        hist.beta.append(beta)
        if callback is not None:
            callback(it, hist.J[-1], hist.G[-1], change, beta)
        if (it + 1) % beta_every == 0 and beta < beta_max:
            beta *= 2.0
            st = MMAState()  # the projected problem changed: restart the asymptotes
        elif change < tol_change and beta >= beta_max:
            break
    with torch.no_grad():
        phys = physical_field(x, mask, R, beta, eta)
    return phys, x, hist
