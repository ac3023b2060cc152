"""GPU: the paper-scale design volume of Fig. 4 -- 621 x 621 x 261 voxels at 177 nm with
absorbing layers [lambda, lambda, 6 lambda] = [6, 6, 36] voxels per face, padded to the FFT
size 640 x 640 x 336 (137.6 M voxels), with a Fresnel lens D = 109 um, NA 0.84, n = 1.54.

Checks, on the full grid:
* the FP64 oracle, at equal iteration count from zero: two forward iterations (the field),
  then two adjoint iterations of |E(r_p)|^2 (the adjoint field) and the gradient.  A
  converged solve here takes ~1e4 iterations, far beyond the oracle's test time, and two
  iterations build the field up only within a few voxels of the plane-wave sheet (after two
  iterations the field falls by about 3x per voxel away from the sheet with this grid's
  shift epsilon = 9.6 k_vac^2), so the objective
  voxel r_p of this check sits one voxel past the sheet, where the field is well above
  rounding;
* at equal iteration count the cuFFT comparison iteration (torch.fft and element-wise torch
  kernels) matches too;
* the gradient and the objective satisfy their definitions on sampled voxels.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2506_15411_gb300 import inputs

pytestmark = pytest.mark.gpu

LAM = 1.064e-6
PITCH = 177e-9
GRID = (640, 640, 336)
PADS = (6, 6, 36)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("CUDA is not available: GPU tests need a GPU")
    return torch


@pytest.fixture(scope="module")
def lens():
    return inputs.fresnel_lens_workload(*GRID, PITCH, LAM, 109e-6, 0.84, 1.54, pad_lo=PADS, pad_hi=PADS)


def _host_memory_gb():
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                return int(ln.split()[1]) / 1e6
    except OSError:
        pass
    return None


@pytest.mark.slow
def test_paper_scale_matches_the_oracle_at_equal_iterations(lens):
    """Field rel-L2 <= 2e-5 and gradient <= 1e-4 against the FP64 oracle after 2 forward and
    2 adjoint iterations from zero on all 137.6 M voxels (objective voxel next to the sheet)."""
    torch = _torch()
    mem = _host_memory_gb()
    if mem is not None and mem < 110:
        pytest.skip(f"the FP64 oracle of this grid needs ~110 GB of host memory ({mem:.0f} GB available)")
    from oracle import cbs_oracle as co
    from paper_2506_15411_gb300 import CBSPlan, PlaneWave
    K = 2
    eps = torch.from_numpy(lens.eps).cuda()
    r0 = (GRID[0] // 2, GRID[1] // 2, lens.z_source + 1)
    with CBSPlan(*GRID, PITCH, LAM, 1.0, PADS, PADS, tol=0.0, max_iter=K, check_every=K) as plan:
        plan.set_permittivity(eps)
        k0g, epg = plan.splitting()
        E, _ = plan.forward(PlaneWave())
        Ea, _ = plan.adjoint(r0, E)
        grad, obj = plan.gradient(E, Ea, r0)
        torch.cuda.synchronize()
        E_h, Ea_h, g_h = E.cpu().numpy(), Ea.cpu().numpy(), grad.cpu().numpy()
    del E, Ea, grad, eps
    torch.cuda.empty_cache()
    g = co.Grid(*GRID, PITCH, LAM, 1.0, PADS, PADS)
    k2 = co.k_squared(g, lens.eps)
    sp = co.splitting(k2)
    assert abs(k0g - sp.k0sq) <= 1e-6 * abs(sp.k0sq) and abs(epg - sp.epsilon) <= 1e-6 * sp.epsilon
    fwd = co.cbs_solve(g, k2, co.plane_wave_source(g), tol=0.0, max_iter=K, split=sp)

    def rel(a, b):
        return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))

    e_fwd = rel(E_h, fwd.E)
    del E_h
    adj = co.cbs_solve(g, k2, co.adjoint_source(g, fwd.E, r0), tol=0.0, max_iter=K, split=sp)
    del k2
    e_adj = rel(Ea_h, adj.E)
    e_grad = rel(g_h, co.gradient(g, fwd.E, adj.E))
    o = co.objective(fwd.E, r0)
    assert e_fwd <= 2e-5, e_fwd
    assert e_adj <= 1e-4, e_adj
    assert e_grad <= 1e-4, e_grad
    assert abs(obj - o) <= 1e-4 * o, (obj, o)


def test_paper_scale_iterations_match_the_cufft_iteration(lens):
    torch = _torch()
    from paper_2506_15411_gb300 import CBSPlan, PlaneWave
    from paper_2506_15411_gb300.cufft_reference import TorchCBS
    K = 4
    eps = torch.from_numpy(lens.eps).cuda()
    with CBSPlan(*GRID, PITCH, LAM, 1.0, PADS, PADS, tol=0.0, max_iter=K, check_every=K) as plan:
        plan.set_permittivity(eps)
        k0sq, epsilon = plan.splitting()
        E, st = plan.forward(PlaneWave())
        torch.cuda.synchronize()
        ref = TorchCBS(eps, PITCH, LAM, 1.0, PADS, PADS, k0sq, epsilon)
        Et = torch.zeros_like(E)
        r = ref.iterate(Et, K)
        torch.cuda.synchronize()
        diff = float(torch.linalg.vector_norm(E - Et) / torch.linalg.vector_norm(Et))
    assert st.iters == K
    assert diff <= 1e-5, diff
    assert abs(float(r) ** 0.5 / st.resid0 - st.rel_resid) <= 1e-4 * st.rel_resid


def test_paper_scale_adjoint_gradient_and_objective(lens):
    torch = _torch()
    from paper_2506_15411_gb300 import CBSPlan, PlaneWave
    K = 8
    eps = torch.from_numpy(lens.eps).cuda()
    r0 = lens.r0
    with CBSPlan(*GRID, PITCH, LAM, 1.0, PADS, PADS, tol=0.0, max_iter=K, check_every=K) as plan:
        plan.set_permittivity(eps)
        E, _ = plan.forward(PlaneWave())
        Ea, sa = plan.adjoint(r0, E)
        grad, obj = plan.gradient(E, Ea, r0)
        torch.cuda.synchronize()
        assert sa.iters == K and torch.isfinite(grad).all()
        x, y, z = r0
        e0 = E[:, z, y, x].cpu().numpy().astype(np.complex128)
        assert abs(obj - float(np.sum(np.abs(e0) ** 2))) <= 1e-6 * obj
        rng = np.random.default_rng(3)
        idx = torch.from_numpy(rng.integers(0, E[0].numel(), 20000)).cuda()
        Ef = E.reshape(3, -1)[:, idx].cpu().numpy().astype(np.complex128)
        Af = Ea.reshape(3, -1)[:, idx].cpu().numpy().astype(np.complex128)
        want = 2 * (2 * np.pi / LAM) ** 2 * np.real(np.sum(Af * Ef, axis=0))
        got = grad.reshape(-1)[idx].cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-6 * np.abs(want).max())
