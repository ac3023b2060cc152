"""Differentiable focal intensity: a torch.autograd.Function over the CUDA CBS solver.

    L(eps_r) = |E(r0)|^2,   E = A(eps_r)^{-1} S,   A = curl curl - k_vac^2 (eps_r + i sigma)

forward runs the CBS forward solve and the objective kernel; backward runs the CBS adjoint
solve (source conj(E(r0)) at r0; A is complex symmetric, so it is the same series) and the
gradient kernel dL/d eps_r = 2 k_vac^2 Re[E_adj . E] -- the adjoint-field method behind the
figure of merit of Fig. 2 and its gradient.  Every step runs in libcbs.so; torch holds the
tensors and chains the gradient into whatever produced eps_r.
"""
from __future__ import annotations

from typing import Optional

import torch

from .solver import CBSPlan, Stats


class FocalIntensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps: torch.Tensor, plan: CBSPlan, source, r0, E_init: Optional[torch.Tensor]):
        eps_c = eps.detach().to(torch.float32).contiguous()
        plan.set_permittivity(eps_c)
        if E_init is not None:
            E, st = plan.forward(source, E=E_init.detach().clone(), warm_start=2)
        else:
            E, st = plan.forward(source)
        r0 = tuple(int(v) for v in r0)
        L = plan.objective(E, r0)
        ctx.plan, ctx.r0, ctx.eps_dtype = plan, r0, eps.dtype
        ctx.save_for_backward(eps_c, E)
        plan.last_forward = st
        plan.last_field = E
        return torch.tensor(L, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, grad_out):
        eps_c, E = ctx.saved_tensors
        plan = ctx.plan
        plan.set_permittivity(eps_c)    # the plan may have solved for another permittivity since
        E_adj, st = plan.adjoint(ctx.r0, E)
        g, _ = plan.gradient(E, E_adj)
        plan.last_adjoint = st
        return (grad_out.to(torch.float32) * g).to(ctx.eps_dtype), None, None, None, None


def focal_intensity(eps: torch.Tensor, plan: CBSPlan, source, r0,
                    E_init: Optional[torch.Tensor] = None) -> torch.Tensor:
    """|E(r0)|^2 (float64 scalar tensor) for the permittivity eps ((nz, ny, nx) on the plan's
    device), differentiable with respect to eps.

    E_init warm-starts the forward series (the fixed point does not depend on it), with the
    residual measured against a start from zero, so a close guess stops early.  After
    the call, plan.last_forward / plan.last_field hold the forward Stats and field, and after
    backward plan.last_adjoint the adjoint Stats; a solve that ends NOT_CONVERGED,
    STAGNATED or TIME_LIMIT does not raise, so callers that need convergence check those
    Stats."""
    return FocalIntensity.apply(eps, plan, source, r0, E_init)


__all__ = ["FocalIntensity", "focal_intensity", "Stats"]
