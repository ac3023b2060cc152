"""GB300-native vector convergent Born series (CBS) solver and adjoint gradient
(arXiv 2506.15411): hand-written sm_103a CUDA behind a C ABI, driven from PyTorch.

`inputs` (seeded synthetic geometry) imports without CUDA; the solver classes load the
compiled library on first use and raise if it is missing.
"""
from __future__ import annotations

__all__ = ["CBSPlan", "PlaneWave", "PointSource", "UserSource", "Stats", "CBSError"]


def __getattr__(name):
    if name in ("CBSPlan", "PlaneWave", "PointSource", "UserSource", "Stats"):
        from . import solver
        return getattr(solver, name)
    if name == "CBSError":
        from ._lib import CBSError
        return CBSError
    raise AttributeError(name)
