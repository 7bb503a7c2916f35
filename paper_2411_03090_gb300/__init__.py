"""GB300-native (sm_103a) Lattice Kinetic Scheme / Adjoint Lattice Kinetic Scheme
for density-based fluid topology optimisation (arXiv 2411.03090).

The compute path is the CUDA library behind ``include/lks.h``; ``lks`` is its
ctypes binding and ``autograd`` wraps gamma -> J as a torch.autograd.Function.
"""
from .lks import (LKS, LKSBatch, LKSError, batch_workspace_size, load, make_desc,  # noqa: F401
                  workspace_size, edge_moment_map)

__all__ = ["LKS", "LKSBatch", "LKSError", "batch_workspace_size", "load", "make_desc", "workspace_size",
           "edge_moment_map"]
