"""The autograd wiring of paper_2506_15411_gb300.autograd on the CPU.

A stand-in plan answers the five plan calls the Function makes with the FP64 oracle (in a
lossy medium k^2 = k_vac^2 (eps_r + 0.3 i) without absorbing layers, where the series
converges in a few hundred iterations; the gradient formula is the same), so the
test checks what the Function itself adds -- the chain rule through torch, the re-setting
of the permittivity before the adjoint, dtypes -- and, through the oracle, that the
backward of |E(r0)|^2 is the adjoint gradient that central differences pin in the oracle's
own tests.  The CUDA path behind the real plan is compared with the oracle in
test_gpu_autograd.py.
"""
from __future__ import annotations

import numpy as np
import torch

from oracle import cbs_oracle as co
from paper_2506_15411_gb300 import inputs
from paper_2506_15411_gb300.autograd import focal_intensity
from paper_2506_15411_gb300.solver import Stats

LAM = 1.064e-6
LOSS = 0.3


class OraclePlan:
    """The subset of CBSPlan the autograd Function uses, answered by the oracle."""

    def __init__(self, grid, S, tol=1e-10):
        self.g, self.S, self.tol = grid, S, tol
        self.eps = None
        self.calls = []

    def set_permittivity(self, eps):
        self.calls.append("set")
        self.eps = eps.double().numpy()

    def _st(self, r):
        return Stats(r.iters, r.rel_resid, r.history[0], 0.0, 0)

    def _solve(self, S):
        return co.cbs_solve(self.g, self.g.k_vac ** 2 * (self.eps + LOSS * 1j), S, tol=self.tol, max_iter=100000)

    def forward(self, source, E=None, warm_start=False):
        self.calls.append("forward")
        r = self._solve(self.S)
        return torch.from_numpy(r.E), self._st(r)

    def objective(self, E, r0):
        return co.objective(E.numpy(), r0)

    def adjoint(self, r0, E):
        self.calls.append("adjoint")
        r = self._solve(co.adjoint_source(self.g, E.numpy(), r0))
        return torch.from_numpy(r.E), self._st(r)

    def gradient(self, E, E_adj):
        return torch.from_numpy(co.gradient(self.g, E.numpy(), E_adj.numpy()).astype(np.float32)), None


def _case():
    g = co.Grid(12, 10, 14, LAM / 6, LAM, 1.0)
    eps = inputs.random_eps(g.nx, g.ny, g.nz, lo=1.0, hi=1.8, seed=31)
    S = co.plane_wave_source(g, z_plane=2)
    return g, eps, S, (6, 5, 10)


def test_backward_is_the_adjoint_gradient_through_the_chain_rule():
    g, eps, S, r0 = _case()
    plan = OraclePlan(g, S)
    p = torch.from_numpy(eps.astype(np.float64)).requires_grad_(True)
    L = focal_intensity(p, plan, None, r0)
    loss = 3.0 * L + L ** 2
    loss.backward()
    assert plan.calls == ["set", "forward", "set", "adjoint"]
    k2 = g.k_vac ** 2 * (eps.astype(np.float64) + LOSS * 1j)
    fwd = co.cbs_solve(g, k2, S, tol=1e-10, max_iter=100000)
    adj = co.cbs_solve(g, k2, co.adjoint_source(g, fwd.E, r0), tol=1e-10, max_iter=100000)
    Lref = co.objective(fwd.E, r0)
    want = (3.0 + 2.0 * Lref) * co.gradient(g, fwd.E, adj.E)
    assert abs(L.item() - Lref) <= 1e-12 * Lref
    assert p.grad.dtype == torch.float64
    np.testing.assert_allclose(p.grad.numpy(), want, rtol=1e-5, atol=1e-6 * np.abs(want).max())


def test_gradient_flows_into_what_produced_the_permittivity():
    """eps = eps_bg + f * (eps_lens - eps_bg): d loss / d f = (eps_lens - eps_bg) dL/d eps."""
    g, eps, S, r0 = _case()
    plan = OraclePlan(g, S)
    f = torch.from_numpy(((eps - 1.0) / 1.25).astype(np.float32)).requires_grad_(True)
    e = 1.0 + 1.25 * f
    focal_intensity(e, plan, None, r0).backward()
    e2 = e.detach().clone().requires_grad_(True)
    focal_intensity(e2, OraclePlan(g, S), None, r0).backward()
    np.testing.assert_allclose(f.grad.numpy(), 1.25 * e2.grad.numpy(), rtol=1e-6)
    assert f.grad.dtype == torch.float32
