"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds problem descriptions and the design-field generator only: no
step of the lattice kinetic scheme or its adjoint lives here.  Both the CUDA
library and the CPU oracle receive what this module produces.

Design field recipe (all 2-D workloads):
  1. u ~ U[0, 1) on the node lattice from numpy's PCG64 ``default_rng(seed)``;
  2. separable Gaussian filter, sigma = ``sigma`` nodes, truncated at 3 sigma,
     reflecting edges;
  3. standardise to z (mean 0, std 1);
  4. gamma = clip(0.5 + 0.5 z, 0, 1);
  5. gamma = 1 on the non-design strips: ``strip`` node columns at the inlet and
     at the outlet, and every edge node.
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict, replace
from typing import List

import numpy as np

T_FIXED = 0
T_FLUX = 1


def _gauss1d(a: np.ndarray, sigma: float, axis: int) -> np.ndarray:
    """Gaussian smoothing along one axis, truncated at 3 sigma, reflecting edges
    (the edge sample is repeated, as in scipy's 'reflect' mode)."""
    r = int(3.0 * sigma + 0.5)
    x = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sigma) ** 2)
    k /= k.sum()
    pad = [(0, 0)] * a.ndim
    pad[axis] = (r, r)
    ap = np.pad(a, pad, mode="symmetric")
    out = np.zeros_like(a)
    n = a.shape[axis]
    for q, kq in enumerate(k):
        sl = [slice(None)] * a.ndim
        sl[axis] = slice(q, q + n)
        out += kq * ap[tuple(sl)]
    return out


def gamma_field(nx: int, ny: int, seed: int, sigma: float = 4.0, strip: int = 4) -> np.ndarray:
    """Seeded smoothed-noise design field, shape (ny, nx), float64 in [0, 1]."""
    rng = np.random.default_rng(seed)
    noise = rng.random((ny, nx))
    s = _gauss1d(_gauss1d(noise, sigma, 0), sigma, 1)
    z = (s - s.mean()) / max(float(s.std()), 1e-300)
    g = np.clip(0.5 + 0.5 * z, 0.0, 1.0)
    g[:, :strip] = 1.0
    g[:, nx - strip:] = 1.0
    g[0, :] = 1.0
    g[-1, :] = 1.0
    g[:, 0] = 1.0
    g[:, -1] = 1.0
    return g


@dataclass
class Problem:
    """One 2-D channel / box problem (lattice units, dx = dt = 1)."""

    nx: int
    ny: int
    nu: float
    alpha_bar: float
    q_alpha: float = 0.1
    u_max: float = 0.05
    pulse_mean: float = 1.0
    pulse_amp: float = 0.0
    pulse_period: float = 0.0
    in_y0: int = 0
    in_y1: int = -1          # -1: ny - 1
    out_y0: int = 1
    out_y1: int = -2         # -2: ny - 2
    rho_out: float = 1.0
    thermal: int = 0
    K_f: float = 0.0
    K_s: float = 0.0
    q_K: float = 0.1
    t_kind: List[int] = field(default_factory=lambda: [T_FIXED, T_FLUX, T_FIXED, T_FLUX])
    t_val: List[float] = field(default_factory=lambda: [0.0, 0.0, 1.0, 0.0])
    kappa_T: float = 0.0
    kappa_p: float = 0.0     # weight of the static pressure drop in J (J = J_O + kappa_p J_p)
    steady: bool = True
    n_steps: int = 1000
    n_adj: int = 1000
    seed: int = 1
    sigma: float = 4.0
    strip: int = 4
    periodic: int = 0        # oracle-only pin geometries: bit 0 x periodic, bit 1 y periodic
    G_x: float = 0.0         # oracle-only pin geometries: uniform external force
    G_y: float = 0.0
    beta_bar: float = 0.0    # heat source Q = beta_gamma (1 - T) (0: none)
    q_beta: float = 0.1
    kappa_Q: float = 0.0     # weight of the heat-exchange objective -sum beta_gamma (1 - T)
    gb_x: float = 0.0        # Boussinesq force G = g beta (T - T_ref): the products g_a beta
    gb_y: float = 0.0
    T_ref: float = 0.0
    heat_x0: int = 0         # heated segment [heat_x0, heat_x1] of a heat-flux bottom edge
    heat_x1: int = -1        # (-1: none)
    heat_q: float = 0.0      # its heat flux
    kappa_E: float = 0.0     # weight of the energy loss J_E (sum of -n.u (p + |u|^2 / 2) over inlet and outlet)

    def resolved(self, name: str):
        """Field value with negative span ends counted from the top edge (ny + v)."""
        v = getattr(self, name)
        if name in ("in_y0", "in_y1", "out_y0", "out_y1") and v < 0:
            return self.ny + v
        return v

    @property
    def n_nodes(self) -> int:
        return self.nx * self.ny

    def gamma(self) -> np.ndarray:
        return gamma_field(self.nx, self.ny, self.seed, self.sigma, self.strip)

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)

    def as_dict(self) -> dict:
        return asdict(self)


def channel(nx: int, ny: int, Re: float, u_max: float = 0.05, **kw) -> Problem:
    """Channel with a parabolic inlet over the whole left edge, pressure outlet on
    the right edge, no-slip walls top and bottom.  nu = u_max L / Re with L the
    inlet width in lattice units (ny - 1); alpha_bar = 1e3 nu."""
    L = ny - 1
    nu = u_max * L / Re
    kw.setdefault("alpha_bar", 1e3 * nu)
    return Problem(nx=nx, ny=ny, nu=nu, u_max=u_max, **kw)


def config1() -> Problem:
    """64x64 steady channel, Re = 10, 5000 forward + 5000 adjoint steps."""
    return channel(64, 64, Re=10.0, seed=1, n_steps=5000, n_adj=5000)


def config2() -> Problem:
    """512x256 steady channel, Re = 100, 20000 forward + 20000 adjoint steps."""
    return channel(512, 256, Re=100.0, seed=2, n_steps=20000, n_adj=20000)


def config3() -> Problem:
    """1024x512 unsteady thermal channel, Re = 200, Pr = 0.71, heated bottom wall,
    pulsed inlet u_max (0.75 + 0.25 sin(2 pi t / 2000)), 20000 steps."""
    p = channel(1024, 512, Re=200.0, seed=3, steady=False, n_steps=20000, n_adj=20000,
                pulse_mean=0.75, pulse_amp=0.25, pulse_period=2000.0, thermal=1,
                kappa_T=1e-4)
    p.K_f = p.nu / 0.71
    p.K_s = p.K_f
    return p


def config5(n_designs: int = 64, n_steps: int = 5000) -> List[Problem]:
    """Batch of unsteady channel designs of unequal size.  Sizes and Reynolds
    numbers come from one generator seeded 5, drawn design by design as
    (nx ~ U{128..512}, ny ~ U{64..256}, Re ~ U[20, 200]); nu = min(0.05 L / Re, 0.30)
    with L = ny - 1 (the clamp keeps nu inside the stable range of the scheme) and
    u_max = Re nu / L; pulsed inlet as config3; design k's gamma uses seed 500 + k."""
    rng = np.random.default_rng(5)
    out = []
    for k in range(n_designs):
        nx = int(rng.integers(128, 513))
        ny = int(rng.integers(64, 257))
        Re = float(rng.uniform(20.0, 200.0))
        L = ny - 1
        nu = min(0.05 * L / Re, 0.30)
        out.append(Problem(nx=nx, ny=ny, nu=nu, alpha_bar=1e3 * nu, u_max=Re * nu / L, steady=False,
                           n_steps=n_steps, n_adj=n_steps, pulse_mean=0.75, pulse_amp=0.25,
                           pulse_period=2000.0, seed=500 + k))
    return out


def gamma_field3(nx: int, ny: int, nz: int, seed: int, sigma: float = 6.0, strip: int = 4) -> np.ndarray:
    """Seeded smoothed-noise design field of a 3-D lattice, shape (nz, ny, nx): the
    2-D recipe with the filter applied along all three axes; gamma = 1 on
    ``strip`` node layers at the inlet and outlet and on every face node."""
    rng = np.random.default_rng(seed)
    noise = rng.random((nz, ny, nx))
    s = _gauss1d(_gauss1d(_gauss1d(noise, sigma, 0), sigma, 1), sigma, 2)
    z = (s - s.mean()) / max(float(s.std()), 1e-300)
    g = np.clip(0.5 + 0.5 * z, 0.0, 1.0)
    g[:, :, :strip] = 1.0
    g[:, :, nx - strip:] = 1.0
    g[0, :, :] = g[-1, :, :] = 1.0
    g[:, 0, :] = g[:, -1, :] = 1.0
    g[:, :, 0] = g[:, :, -1] = 1.0
    return g


@dataclass
class Problem3:
    """One 3-D (D3Q19) steady duct: inlet face x = 0, outlet face x = nx - 1, walls
    on the four side faces (lattice units)."""

    nx: int
    ny: int
    nz: int
    nu: float
    alpha_bar: float
    q_alpha: float = 0.1
    u_max: float = 0.05
    rho_out: float = 1.0
    profile: int = 0         # inlet: 0 duct (product of parabolas), 1 plane channel (parabola in y)
    kappa_p: float = 0.0     # weight of the static pressure drop in J (J = J_O + kappa_p J_p)
    steady: bool = True
    n_steps: int = 1000
    n_adj: int = 1000
    seed: int = 4
    sigma: float = 6.0
    strip: int = 4

    @property
    def n_nodes(self) -> int:
        return self.nx * self.ny * self.nz

    def gamma(self) -> np.ndarray:
        return gamma_field3(self.nx, self.ny, self.nz, self.seed, self.sigma, self.strip)

    def with_(self, **kw) -> "Problem3":
        return replace(self, **kw)


def duct(nx: int, ny: int, nz: int, Re: float, u_max: float = 0.05, **kw) -> Problem3:
    """Duct with the inlet over the whole x = 0 face; nu = u_max L / Re with L the
    inlet width ny - 1; alpha_bar = 1e3 nu."""
    nu = u_max * (ny - 1) / Re
    kw.setdefault("alpha_bar", 1e3 * nu)
    return Problem3(nx=nx, ny=ny, nz=nz, nu=nu, u_max=u_max, **kw)


def config4() -> Problem3:
    """192^3 steady duct, Re = 50 (nu = 0.191), sigma = 6, 1000 forward + 1000
    adjoint steps; J = total dissipation + static pressure drop (unit weights)."""
    return duct(192, 192, 192, Re=50.0, seed=4, n_steps=1000, n_adj=1000, kappa_p=1.0)


def roofline2d(n: int = 8192) -> Problem:
    """Large 2-D steady channel used to load HBM (working set >> L2)."""
    return channel(n, n, Re=100.0 * (n - 1) / 255.0, seed=6, n_steps=200, n_adj=200)


def natural_convection_cavity(scale: float = 0.5, Ra: float = 2e4, Pr: float = 0.71, nu: float = 0.06,
                              q0: float = 1e-2, kappa_T: float = 1e-3, n_steps: int = 2000) -> tuple:
    """The natural-convection sensitivity check of Sec. 2.6 (its verification of the
    natural convection problem): a closed 140 x 80 (dx) cavity of walls, scaled by
    `scale`; T = 0 prescribed on the left, right and top walls; the bottom wall
    adiabatic except a heated centre part of 4 dx (heat flux q0); gravity along -y
    with the Boussinesq force G = g beta (T - 0), g beta from Ra = g beta L^3 / (nu K_f)
    with L the cavity height and Delta T = 1; K_s = 10 K_f.  The design domain is the
    central 80 x 50, gamma = 0.1 in its central 40 x 25 and 0.9 elsewhere in it, and
    gamma = 1 (fluid) outside.  The objective is kappa_T times the sum of T over the
    interior nodes (the paper does not state the check's objective).
    Returns (problem, gamma)."""
    nx, ny = int(round(140 * scale)) + 1, int(round(80 * scale)) + 1
    L = ny - 1
    K_f = nu / Pr
    gb = Ra * nu * K_f / L ** 3
    cx = (nx - 1) // 2
    hw = max(1, int(round(2 * scale)))
    pb = Problem(nx=nx, ny=ny, nu=nu, alpha_bar=1e3 * nu, u_max=0.0, in_y0=0, in_y1=ny - 1, out_y0=1, out_y1=0,
                 thermal=1, K_f=K_f, K_s=10.0 * K_f, t_kind=[T_FIXED, T_FIXED, T_FLUX, T_FIXED],
                 t_val=[0.0, 0.0, 0.0, 0.0], heat_x0=cx - hw, heat_x1=cx + hw, heat_q=q0, gb_x=0.0, gb_y=-gb,
                 T_ref=0.0, kappa_T=kappa_T, n_steps=n_steps, n_adj=n_steps)
    g = np.ones((ny, nx))
    y, x = np.mgrid[0:ny, 0:nx]
    dx0, dx1 = int(round(30 * scale)), int(round(110 * scale))
    dy0, dy1 = int(round(15 * scale)), int(round(65 * scale))
    g[(x >= dx0) & (x <= dx1) & (y >= dy0) & (y <= dy1)] = 0.9
    ix0, ix1 = int(round(50 * scale)), int(round(90 * scale))
    iy0, iy1 = int(round(27.5 * scale)), int(round(52.5 * scale))
    g[(x >= ix0) & (x <= ix1) & (y >= iy0) & (y <= iy1)] = 0.1
    return pb, g


def forced_convection_check(n: int = 31, Pr: float = 0.71, beta_bar: float = 0.01, nu: float = 0.1,
                            kappa_Q: float = 1.0, n_steps: int = 40000) -> tuple:
    """The forced-convection sensitivity check of Sec. 2.6 on the domain of its
    non-thermal check, at n x n nodes: walls, a parabolic inlet over the middle third
    of the left edge and an outlet over the same rows of the right edge, nu = 0.1,
    Re = 1 on the inlet width; gamma = 0.1 in the centre circle of radius n / 6 and
    0.9 elsewhere.  T = 0 is prescribed on the inlet (left) edge and every other edge
    is adiabatic.  The solid heats the fluid through the source Q = beta_gamma (1 - T)
    (Eqs. heatsource, betagamma) and J adds the heat-exchange objective
    -kappa_Q sum beta_gamma (1 - T) (Eq. objective_heatexchanger) to the dissipation.
    Unstated and chosen: Pr, beta_bar, K_s = K_f.  Returns (problem, gamma)."""
    a, b = (n - 1) // 3, 2 * (n - 1) // 3
    K = nu / Pr
    pb = Problem(nx=n, ny=n, nu=nu, alpha_bar=1e3 * nu, u_max=nu / (b - a), in_y0=a, in_y1=b, out_y0=a, out_y1=b,
                 thermal=1, K_f=K, K_s=K, t_kind=[T_FIXED, T_FLUX, T_FLUX, T_FLUX], t_val=[0.0, 0.0, 0.0, 0.0],
                 beta_bar=beta_bar, kappa_Q=kappa_Q, n_steps=n_steps, n_adj=n_steps)
    c = (n - 1) / 2.0
    yy, xx = np.mgrid[0:n, 0:n]
    g = np.where((xx - c) ** 2 + (yy - c) ** 2 <= (n / 6.0) ** 2, 0.1, 0.9)
    return pb, g


def poiseuille(nx: int = 33, ny: int = 17, nu: float = 0.1, u_max: float = 0.02) -> Problem:
    """Empty channel (gamma = 1 everywhere) for the Poiseuille pin."""
    return Problem(nx=nx, ny=ny, nu=nu, alpha_bar=1e3 * nu, u_max=u_max)
