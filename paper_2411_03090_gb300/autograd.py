"""gamma -> J as a torch.autograd.Function whose backward is the ALKS march.

Forward: Steps 2-3 of the paper's procedure (Sec. 2.7) through ``lks_forward``.
Backward: Steps 4-5 through ``alks_adjoint`` and ``lks_sensitivity``, scaled by the
incoming gradient of J.
"""
from __future__ import annotations

import torch

from .lks import LKS


class LKSObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gamma: torch.Tensor, solver: LKS) -> torch.Tensor:
        J = solver.lks_forward(gamma.detach()).clone()
        ctx.solver = solver
        ctx.gamma_dtype = gamma.dtype
        return J

    @staticmethod
    def backward(ctx, grad_J: torch.Tensor):
        s: LKS = ctx.solver
        s.alks_adjoint()
        g = s.lks_sensitivity()
        return (grad_J.to(g.dtype) * g).to(ctx.gamma_dtype), None


def objective(gamma: torch.Tensor, solver: LKS) -> torch.Tensor:
    """J(gamma) with the ALKS gradient attached."""
    return LKSObjective.apply(gamma, solver)
