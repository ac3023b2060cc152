"""GPU: torch.autograd through the CUDA forward solve, adjoint solve and gradient kernel.

1. Equal iterations against the FP64 oracle on a small design-slab grid: the objective and
   dL/d eps_r (chained through a scalar loss) to relative L2 1e-4 / 1e-3.
2. Central finite differences on 32 random voxels of a design slab (seed 7), on a 96x96x64
   grid and on the 256x256x192 design volume of item 3 (there with gentler absorbing layers,
   see FD_CASES).  A single-voxel
   change moves |E(r0)|^2 by ~1e-4 of itself, below what two FP32 solves resolve when
   differenced; so each side is computed through the field change instead:
   E_+- = E + D_+-, with (curl curl - k_+-^2) D_+- = (k_+-^2 - k^2) E = +-h k_vac^2 E(r) at
   voxel r -- an exact identity, solved by the same CBS as a point source -- and
   L_+ - L_- = 2 Re[conj(E(r0)).(D_+ - D_-)] + |D_+|^2 - |D_-|^2 in FP64.
3. The 256x256x192 design volume at lambda/8 (slab 192x192x48): a directional central
   difference of L, from plain forward solves, along the gradient on a random half of the
   slab's voxels.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import cbs_oracle as co
from paper_2506_15411_gb300 import inputs

pytestmark = pytest.mark.gpu

LAM = 1.064e-6


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("CUDA is not available: GPU tests need a GPU")
    return torch


def _design_case(nx, ny, nz, pitch, slab, pads, z_gap=2):
    """Design slab above the plane-wave sheet; focus f_eff above the slab base, D = slab width."""
    z_base = pads[2] + z_gap
    D = slab[0] * pitch
    eps, region = inputs.design_slab_eps(nx, ny, nz, pitch, LAM, slab=slab, D=D, z_base=z_base)
    zf = z_base + int(round(inputs.focal_length(D, 0.84) / pitch))
    assert zf < nz - pads[2]
    return eps, region, (nx // 2, ny // 2, zf)


def test_autograd_matches_oracle_at_equal_iterations():
    torch = _torch()
    from paper_2506_15411_gb300 import CBSPlan, PlaneWave
    from paper_2506_15411_gb300.autograd import focal_intensity
    nx, ny, nz, pitch, pads = 40, 36, 48, LAM / 8, (4, 4, 6)
    eps, region, r0 = _design_case(nx, ny, nz, pitch, (24, 20, 8), pads)
    K = 300
    g = co.Grid(nx, ny, nz, pitch, LAM, 1.0, pads, pads)
    fwd = co.forward(g, eps, co.plane_wave_source(g), tol=0.0, max_iter=K)
    adj = co.adjoint(g, eps, fwd.E, r0, tol=0.0, max_iter=K)
    L_ref = co.objective(fwd.E, r0)
    g_ref = 2.5 * co.gradient(g, fwd.E, adj.E)
    with CBSPlan(nx, ny, nz, pitch, LAM, 1.0, pads, pads, tol=0.0, max_iter=K, check_every=50) as plan:
        e = torch.from_numpy(eps).cuda().requires_grad_(True)
        L = focal_intensity(e, plan, PlaneWave(), r0)
        (2.5 * L).backward()
        torch.cuda.synchronize()
        assert plan.last_forward.iters == K and plan.last_adjoint.iters == K
    assert abs(L.item() - L_ref) <= 1e-4 * L_ref
    gg = e.grad.cpu().numpy()
    assert np.linalg.norm(gg - g_ref) <= 1e-3 * np.linalg.norm(g_ref)
    assert np.linalg.norm((gg - g_ref)[region]) <= 1e-3 * np.linalg.norm(g_ref[region])


def _field_change_fd(plan, eps_dev, E, r0, v, h):
    """(L(eps + h e_v) - L(eps - h e_v)) / 2h through the field change (module docstring).
    The minus side starts from -D_+, which it equals to first order in h.  Returns the
    difference and the two solves' iteration counts."""
    import torch
    from paper_2506_15411_gb300 import PointSource
    x, y, z = v
    Ev = E[:, z, y, x].cpu().numpy().astype(np.complex128)
    E0 = E[:, r0[2], r0[1], r0[0]].cpu().numpy().astype(np.complex128)
    kv2 = (2 * np.pi / plan.lam) ** 2
    L, iters, Dp = [], [], None
    for s in (+1.0, -1.0):
        e = eps_dev.clone()
        e[z, y, x] += s * h
        plan.set_permittivity(e)
        src = PointSource(v, tuple(s * h * kv2 * Ev))
        if Dp is None:
            D, st = plan.forward(src)
            Dp = D.clone()
        else:
            D, st = plan.forward(src, E=-Dp, warm_start=2)
        assert st.converged, st
        iters.append(st.iters)
        Dr = D[:, r0[2], r0[1], r0[0]].cpu().numpy().astype(np.complex128)
        L.append(2 * np.real(np.vdot(E0, Dr)) + np.sum(np.abs(Dr) ** 2))
    plan.set_permittivity(eps_dev)
    torch.cuda.synchronize()
    return (L[0] - L[1]) / (2 * h), iters


# (grid, slab, pads, layer options): a 96x96x64 slab grid, and the 256x256x192 design volume
# at lambda/8 with its 192x192x48 slab.  On the design volume the default layers make each
# field-change solve about 27 000 iterations (64 of them: 13 minutes of GPU time); the gentler
# setting (round trip 1e-2, largest profile in the corners) takes about 6 500.  The identity
# checked -- the adjoint gradient against differences of L -- holds for any absorbing profile,
# and both sides of it see the same one.
GENTLE = dict(layer_round_trip=1e-2, layer_corner_max=True)
FD_CASES = {
    "slab_96x96x64": ((96, 96, 64), (64, 64, 16), (8, 8, 12), {}),
    "design_volume_256x256x192": ((256, 256, 192), (192, 192, 48), (8, 8, 24), GENTLE),
}


@pytest.mark.parametrize("case", list(FD_CASES))
def test_autograd_central_differences_on_random_slab_voxels(case):
    import time
    torch = _torch()
    from paper_2506_15411_gb300 import CBSPlan, PlaneWave
    from paper_2506_15411_gb300.autograd import focal_intensity
    (nx, ny, nz), slab, pads, layers = FD_CASES[case]
    pitch = LAM / 8
    eps, region, r0 = _design_case(nx, ny, nz, pitch, slab, pads)
    rng = np.random.default_rng(7)
    zs, ys, xs = (rng.integers(s.start, s.stop, 32) for s in region)
    t0 = time.perf_counter()
    with CBSPlan(nx, ny, nz, pitch, LAM, 1.0, pads, pads, tol=3e-5, max_iter=100000, check_every=32,
                 **layers) as plan:
        e = torch.from_numpy(eps).cuda().requires_grad_(True)
        L = focal_intensity(e, plan, PlaneWave(), r0)
        L.backward()
        E = plan.last_field
        grad = e.grad.cpu().numpy()
        assert plan.last_forward.converged and plan.last_adjoint.converged
        it_fa = (plan.last_forward.iters, plan.last_adjoint.iters)
        plan.set_solver(1e-4, 100000, 32)
        h = 0.05
        res = [_field_change_fd(plan, e.detach(), E, r0, (int(x), int(y), int(z)), h)
               for x, y, z in zip(xs, ys, zs)]
    fd = np.array([r[0] for r in res])
    it_fd = np.array([r[1] for r in res])
    print(f"{case}: forward/adjoint iterations {it_fa}, field-change solves {it_fd[:, 0].mean():.0f} (+) "
          f"{it_fd[:, 1].mean():.0f} (-, warm) on average, {time.perf_counter() - t0:.1f} s")
    gs = grad[zs, ys, xs]
    scale = np.abs(fd).max()
    assert scale > 0
    # FD truncation (h^2 terms of a single-voxel rational dependence) and FP32 solves
    err = np.abs(gs - fd)
    assert np.all(err <= 1e-2 * np.abs(fd) + 1e-3 * scale), np.max(err / (np.abs(fd) + 0.1 * scale))


def test_autograd_design_volume_directional_difference():
    torch = _torch()
    from paper_2506_15411_gb300 import CBSPlan, PlaneWave
    from paper_2506_15411_gb300.autograd import focal_intensity
    nx, ny, nz, pitch, pads = 256, 256, 192, LAM / 8, (8, 8, 24)
    eps, region, r0 = _design_case(nx, ny, nz, pitch, (192, 192, 48), pads)
    rng = np.random.default_rng(7)
    mask = np.zeros(eps.shape, dtype=bool)
    mask[region] = rng.random(mask[region].shape) < 0.5
    tol = 1e-4
    with CBSPlan(nx, ny, nz, pitch, LAM, 1.0, pads, pads, tol=tol, max_iter=100000, check_every=64) as plan:
        e = torch.from_numpy(eps).cuda().requires_grad_(True)
        L = focal_intensity(e, plan, PlaneWave(), r0)
        L.backward()
        E = plan.last_field
        assert plan.last_forward.rel_resid <= tol and plan.last_adjoint.rel_resid <= tol
        g = e.grad.cpu().numpy().astype(np.float64)
        # direction: the gradient on a random half of the slab (a random +-1 pattern cancels
        # to a slope too small for a difference of FP32 solves to resolve)
        d = np.where(mask, g, 0.0) / np.abs(g[mask]).max()
        slope = float(np.sum(g * d))
        L0 = L.item()
        h = 0.05 * L0 / abs(slope)      # moves L by about 5 % each way
        assert h <= 0.1, h
        dd = torch.from_numpy(d.astype(np.float32)).cuda()
        Ls = []
        for s in (+1.0, -1.0):
            with torch.no_grad():
                Ls.append(focal_intensity(e.detach() + s * h * dd, plan, PlaneWave(), r0, E_init=E).item())
            assert plan.last_forward.converged, plan.last_forward
    fd = (Ls[0] - Ls[1]) / (2 * h)
    assert abs(fd - slope) <= 1e-2 * abs(slope), (fd, slope, L0, h)
