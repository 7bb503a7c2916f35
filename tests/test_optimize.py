"""The optimisation loop of Sec. 2.7 (Steps 1-7): MMA, filter, projection, loop.

CPU tests check each piece against a closed form or torch's own autograd; the GPU
test runs a few design iterations of a small channel through the CUDA library.
"""
import math

import numpy as np
import pytest
import torch

from paper_2411_03090_gb300.optimize import (MMAState, density_filter, heaviside_projection, mma_update,
                                             optimize, physical_field)


def test_mma_reaches_the_kkt_point_of_a_convex_problem():
    """min sum_j c_j / x_j  s.t.  mean(x) <= V,  1e-3 <= x <= 1: the constraint binds
    and the optimum is x_j = n V sqrt(c_j) / sum_k sqrt(c_k) (Lagrange condition
    c_j / x_j^2 = const)."""
    g = torch.Generator().manual_seed(3)
    n, V = 200, 0.3
    c = 0.5 + torch.rand(n, generator=g, dtype=torch.float64)
    exact = n * V * torch.sqrt(c) / torch.sqrt(c).sum()
    assert float(exact.max()) < 1.0
    x = torch.full((n,), V, dtype=torch.float64)
    st = MMAState()
    for _ in range(60):
        f0g = -c / x ** 2
        f1 = float(x.mean()) - V
        f1g = torch.full_like(x, 1.0 / n)
        x = mma_update(x, f0g, f1, f1g, st, xmin=1e-3, xmax=1.0)
    assert float((x - exact).abs().max()) < 1e-5
    assert float(x.mean()) - V < 1e-9


def test_mma_with_an_inactive_constraint():
    """min sum_j (c_j / x_j + x_j) with mean(x) far below the bound: the constraint
    does not bind (multiplier zero) and MMA converges to x_j = sqrt(c_j).  The
    asymptotes may not come closer than asymin times the range to x; with the usual
    0.01 the iterates settle within about that distance, with 1e-6 to round-off."""
    g = torch.Generator().manual_seed(4)
    c = 0.01 + 0.05 * torch.rand(50, generator=g, dtype=torch.float64)
    for asymin, tol in ((1e-2, 2e-2), (1e-6, 1e-12)):
        x = torch.full_like(c, 0.5)
        st = MMAState()
        for _ in range(200):
            x = mma_update(x, -c / x ** 2 + 1.0, float(x.mean()) - 0.9, torch.full_like(x, 1 / 50), st,
                           xmin=1e-3, asymin=asymin)
        assert float((x - torch.sqrt(c)).abs().max()) < tol


def test_density_filter_is_a_normalised_cone_average():
    """Constant fields are preserved (weights normalised at every node, also at the
    edges), and an interior value equals the cone-weighted average written out."""
    R = 2.4
    x = torch.rand(12, 15, dtype=torch.float64, generator=torch.Generator().manual_seed(5))
    np.testing.assert_allclose(density_filter(torch.full((12, 15), 0.7, dtype=torch.float64), R).numpy(), 0.7,
                               rtol=0, atol=1e-15)
    out = density_filter(x, R)
    for (j, i) in [(6, 7), (0, 0), (11, 3)]:
        num = den = 0.0
        for jj in range(12):
            for ii in range(15):
                w = max(0.0, R - math.hypot(jj - j, ii - i))
                num += w * float(x[jj, ii])
                den += w
        assert abs(float(out[j, i]) - num / den) < 1e-14


def test_heaviside_projection_endpoints_and_limit():
    """H(0) = 0, H(1) = 1, H(eta) = tanh(beta eta) / (tanh(beta eta) + tanh(beta (1 - eta)))
    (1/2 at eta = 1/2), monotone, and a step at eta for large beta."""
    xs = torch.linspace(0, 1, 101, dtype=torch.float64)
    for beta in (1.0, 8.0, 64.0):
        h = heaviside_projection(xs, beta)
        assert abs(float(h[0])) < 1e-15 and abs(float(h[-1]) - 1) < 1e-15
        assert abs(float(h[50]) - 0.5) < 1e-15
        assert bool((h[1:] >= h[:-1]).all())
    h = heaviside_projection(torch.tensor([0.45, 0.55], dtype=torch.float64), 512.0)
    assert float(h[0]) < 1e-6 and float(h[1]) > 1 - 1e-6


def test_loop_on_a_separable_objective():
    """The loop (filter, projection, MMA, beta continuation) on a smooth objective
    that prefers fluid along the centre line: J falls, the area constraint holds at
    the end, and nodes outside the design domain stay at gamma = 1."""
    ny, nx = 20, 30
    yy, _ = torch.meshgrid(torch.arange(ny, dtype=torch.float64), torch.arange(nx, dtype=torch.float64),
                           indexing="ij")
    w = torch.exp(-((yy - 10) ** 2) / 20.0)
    mask = torch.zeros(ny, nx, dtype=torch.bool)
    mask[2:-2, 3:-3] = True

    def J_of(gamma):
        return (w / (gamma + 0.05)).sum()

    phys, x, hist = optimize(J_of, mask, vmax=0.4, n_iter=60, R=1.5, beta0=1.0, beta_every=20, beta_max=8.0)
    assert hist.J[-1] < 0.95 * hist.J[0]
    assert hist.G[-1] <= 1e-3
    assert bool((phys[~mask] == 1).all())
    assert float(phys[mask].mean()) <= 0.4 + 1e-3


@pytest.mark.gpu
def test_loop_on_the_gpu_channel():
    """Steps 1-7 on a 48 x 32 channel through the CUDA library (FP32, steady,
    warm-started marches, dissipation objective): after 12 iterations J is below its
    first value and the area constraint holds to 1e-3."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import inputs
    from paper_2411_03090_gb300 import LKS
    from paper_2411_03090_gb300.autograd import objective

    pb = inputs.channel(48, 32, Re=10.0, n_steps=600, n_adj=600)
    s = LKS(pb, real="f32", warm_start=True)
    mask = torch.zeros(pb.ny, pb.nx, dtype=torch.bool, device="cuda")
    mask[1:-1, 6:-6] = True
    phys, x, hist = optimize(lambda g: objective(g, s), mask, vmax=0.5, n_iter=12, R=2.4, beta0=1.0)
    assert all(np.isfinite(hist.J))
    assert min(hist.J[1:]) < hist.J[0]
    assert hist.G[-1] <= 1e-3
    assert s.query().device_status == 0
