"""GPU: the design step of Section 3 / Fig. 2(a) (cbs_design_*) against the FP64 design oracle.

The surface voxel of a pixel is floor(h_eff / pitch), an integer decided by floating point;
the GPU forms h_eff in FP32 and the oracle in FP64, so a pixel whose h_eff sits within
1e-3 voxel of a voxel face may pick the other voxel.  The kernel test feeds the GPU's own
h_eff to the oracle's chain rule (then only the rounding of h_eff / pitch separates the
decisions); the full step compares on pixels that no ambiguous pixel can reach through the
smoothing and the mirror average: at least half of the map with the Gaussian filter, and at
least 99 % without it (sigma = 0), where a pixel's reach is itself and its mirror images.
The fill fraction keeps eps continuous in h, so a flipped decision changes only the surface
derivative of the pixels it reaches, not the field.  Each case prints its ambiguous-pixel
count.  Adam's first step is alpha * g / (|g| + eps)
~ alpha sign(g): where |dL/dh| is below 1e-3 of its maximum the sign is not resolved by an
FP32 gradient, and there the check is that the step is valid (|dh| <= alpha, within the box).
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import cbs_oracle as co
from oracle import design as od
from paper_2506_15411_gb300 import inputs

pytestmark = pytest.mark.gpu

LAM = 1.064e-6


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("CUDA is not available: GPU tests need a GPU")
    return torch


def _case(sigma_um=0.355, mirror=True):
    nx, ny, nz, pitch, pads = 40, 40, 36, LAM / 8, (4, 4, 6)
    p_um = pitch * 1e6
    z_base = pads[2] + 2
    D_um = 24 * p_um
    prm = od.DesignParams(z_base=z_base, n_lens=1.5, aperture_um=D_um, h_max_um=LAM * 1e6 / 0.5,
                          sigma_um=sigma_um, mirror=mirror)
    x = inputs.centred_coords(nx, p_um)
    y = inputs.centred_coords(ny, p_um)
    r = np.sqrt(x[None, :] ** 2 + y[:, None] ** 2)
    h0 = inputs.fresnel_height(r, LAM * 1e6, D_um, 0.84, 1.5)       # micrometres
    zf = z_base + int(round(inputs.focal_length(D_um, 0.84) / p_um))
    grid = co.Grid(nx, ny, nz, pitch, LAM, 1.0, pads, pads)
    return grid, prm, h0.astype(np.float32), (nx // 2, ny // 2, zf)


def _design(plan, prm):
    from paper_2506_15411_gb300.design import Design
    return Design(plan, prm.z_base, prm.n_lens, prm.aperture_um, prm.h_max_um, prm.sigma_um, prm.mirror,
                  prm.alpha, prm.beta1, prm.beta2, prm.adam_eps)


def _trusted_pixels(h_eff_oracle, p_um, prm, tol=1e-3, label=""):
    """Pixels whose dL/dh cannot depend on an ambiguous surface voxel (u within tol of a face
    above the base; u ~ 0 is not ambiguous, h_eff >= 0 on both sides)."""
    u = od.surface_coordinate(h_eff_oracle, p_um)
    amb = (np.abs(u - np.round(u)) < tol) & (np.round(u) >= 1)
    print(f"{label} sigma={prm.sigma_um} mirror={prm.mirror}: {int(amb.sum())} ambiguous pixels "
          f"of {amb.size} (tol {tol:g} voxel)")
    R = int(np.ceil(4 * prm.sigma_um / p_um)) if prm.sigma_um > 0 else 0
    reach = np.zeros_like(amb)
    for y, x in zip(*np.nonzero(amb)):
        reach[max(0, y - R):y + R + 1, max(0, x - R):x + R + 1] = True
    if prm.mirror:
        reach = reach | reach[::-1, :] | reach[:, ::-1] | reach[::-1, ::-1]
    return ~reach


@pytest.mark.parametrize("sigma_um,mirror", [(0.355, True), (0.0, False)])
def test_pipeline_kernels_match_oracle(sigma_um, mirror):
    torch = _torch()
    from paper_2506_15411_gb300 import CBSPlan
    g, prm, h0, _ = _case(sigma_um, mirror)
    p_um = g.pitch * 1e6
    rng = np.random.default_rng(12)
    h = (h0 + rng.uniform(0, 0.2, h0.shape)).astype(np.float32)      # not symmetric
    grad_eps = rng.standard_normal(g.shape).astype(np.float32)
    with CBSPlan(g.nx, g.ny, g.nz, g.pitch, LAM, 1.0, g.pad_lo, g.pad_hi) as plan:
        with _design(plan, prm) as d:
            hd = torch.from_numpy(h).cuda()
            eps, he = d.permittivity(hd)
            gh = d.height_gradient(hd, torch.from_numpy(grad_eps).cuda())
            torch.cuda.synchronize()
    he_ref = od.effective_height(h.astype(np.float64), p_um, prm)
    np.testing.assert_allclose(he.cpu().numpy(), he_ref, rtol=0, atol=2e-6)
    eps_ref = od.permittivity(he_ref, g.nz, p_um, prm.z_base, prm.n_lens, 1.0)
    np.testing.assert_allclose(eps.cpu().numpy(), eps_ref, rtol=0, atol=2e-5)
    if mirror:       # the mirror average and the paired filter sums keep exact symmetry
        hg = he.cpu().numpy()
        assert np.array_equal(hg, hg[::-1, :]) and np.array_equal(hg, hg[:, ::-1])
    # the surface voxels from the GPU's own h_eff: only FP32 rounding of h_eff / pitch (~1e-6
    # voxel) separates the two decisions
    he_gpu = he.cpu().numpy().astype(np.float64)
    gh_ref = od.height_gradient(grad_eps.astype(np.float64), he_gpu, p_um, prm, 1.0)
    ok = _trusted_pixels(he_gpu, p_um, prm, tol=1e-5, label="kernels")
    assert ok.mean() >= (0.99 if sigma_um == 0 else 0.5)
    err = np.abs(gh.cpu().numpy() - gh_ref)[ok]
    assert np.max(err) <= 1e-5 * np.abs(gh_ref).max()


@pytest.mark.parametrize("sigma_um,mirror,min_trusted", [(0.355, True, 0.5), (0.0, True, 0.99),
                                                       (0.0, False, 0.99)])
def test_design_step_matches_oracle_at_equal_iterations(sigma_um, mirror, min_trusted):
    torch = _torch()
    from paper_2506_15411_gb300 import CBSPlan, PlaneWave
    g, prm, h0, r0 = _case(sigma_um, mirror)
    p_um = g.pitch * 1e6
    K = 300
    st = od.AdamState.zeros(h0.shape)
    ref = od.design_step(g, h0.astype(np.float64), st, prm, co.plane_wave_source(g), r0, tol=0.0, max_iter=K)
    with CBSPlan(g.nx, g.ny, g.nz, g.pitch, LAM, 1.0, g.pad_lo, g.pad_hi, tol=0.0, max_iter=K,
                 check_every=50) as plan:
        with _design(plan, prm) as d:
            h = torch.from_numpy(h0.copy()).cuda()
            gh = torch.empty_like(h)
            info = d.step(h, PlaneWave(), r0, grad_h=gh)
            torch.cuda.synchronize()
            h1, gh1 = h.cpu().numpy(), gh.cpu().numpy()
    assert info.fwd.iters == K and info.adj.iters == K
    assert abs(info.objective - ref.objective) <= 1e-4 * ref.objective
    ok = _trusted_pixels(ref.h_eff, p_um, prm, label="step")
    assert ok.mean() >= min_trusted, ok.mean()
    gmax = np.abs(ref.grad_h).max()
    assert np.linalg.norm((gh1 - ref.grad_h)[ok]) <= 1e-3 * np.linalg.norm(ref.grad_h[ok])
    mask = od.aperture(g.nx, g.ny, p_um, prm.aperture_um)
    assert np.all(h1[~mask] == 0.0)
    strong = ok & mask & (np.abs(ref.grad_h) > 1e-3 * gmax)
    assert strong.sum() >= 0.3 * mask.sum()
    np.testing.assert_allclose(h1[strong], ref.h[strong], rtol=0, atol=1e-5)
    weak = mask & ~strong
    assert np.all(np.abs(h1[weak] - h0[weak]) <= prm.alpha * (1 + 1e-5))
    assert h1.min() >= 0.0 and h1.max() <= prm.h_max_um
    if mirror:
        assert np.array_equal(h1, h1[::-1, :]) and np.array_equal(h1, h1[:, ::-1])


def test_warm_started_steps_converge_to_the_same_result_in_fewer_iterations():
    torch = _torch()
    from paper_2506_15411_gb300 import CBSPlan, PlaneWave
    g, prm, h0, r0 = _case()
    tol = 1e-4
    res = {}
    for warm in (0, 2):
        with CBSPlan(g.nx, g.ny, g.nz, g.pitch, LAM, 1.0, g.pad_lo, g.pad_hi, tol=tol, max_iter=50000,
                     check_every=16) as plan:
            with _design(plan, prm) as d:
                h = torch.from_numpy(h0.copy()).cuda()
                infos = d.run(h, PlaneWave(), r0, steps=3, warm_start=warm)
                torch.cuda.synchronize()
                res[warm] = (h.cpu().numpy(), infos)
    # the first step is the same cold solve; later steps may differ where an Adam sign
    # flips on a gradient below the solves' accuracy
    for k, rtol in ((0, 0.0), (1, 1e-2), (2, 1e-2)):
        a, b = res[0][1][k], res[2][1][k]
        assert a.fwd.converged and b.fwd.converged and a.adj.converged and b.adj.converged
        assert abs(a.objective - b.objective) <= rtol * a.objective, (k, a.objective, b.objective)
    it0 = sum(i.fwd.iters + i.adj.iters for i in res[0][1][1:])
    it2 = sum(i.fwd.iters + i.adj.iters for i in res[2][1][1:])
    assert it2 < it0, (it0, it2)


def test_height_autograd_composes_with_focal_intensity():
    torch = _torch()
    from paper_2506_15411_gb300 import CBSPlan, PlaneWave
    from paper_2506_15411_gb300.autograd import focal_intensity
    from paper_2506_15411_gb300.design import height_to_permittivity
    g, prm, h0, r0 = _case()
    K = 200
    with CBSPlan(g.nx, g.ny, g.nz, g.pitch, LAM, 1.0, g.pad_lo, g.pad_hi, tol=0.0, max_iter=K,
                 check_every=50) as plan:
        with _design(plan, prm) as d:
            h = torch.from_numpy(h0.copy()).cuda().requires_grad_(True)
            L = focal_intensity(height_to_permittivity(h, d), plan, PlaneWave(), r0)
            L.backward()
            hs = torch.from_numpy(h0.copy()).cuda()
            gh = torch.empty_like(hs)
            info = d.step(hs, PlaneWave(), r0, grad_h=gh)
            torch.cuda.synchronize()
    assert abs(L.item() - info.objective) <= 1e-6 * info.objective
    np.testing.assert_allclose(h.grad.cpu().numpy(), gh.cpu().numpy(), rtol=0,
                               atol=1e-6 * float(gh.abs().max()))


def test_checkpoint_and_resume_continue_the_loop_exactly(tmp_path):
    """Two steps, a checkpoint (h, Adam's moments and step count, the fields), two more steps;
    a fresh plan and design object resumed from the file reproduce the last two steps bit for
    bit.  The moments also come back through host pointers."""
    import ctypes
    import dataclasses
    torch = _torch()
    from paper_2506_15411_gb300 import CBSPlan, PlaneWave
    g, prm, h0, r0 = _case()
    path = str(tmp_path / "design.pt")

    def plan():
        return CBSPlan(g.nx, g.ny, g.nz, g.pitch, LAM, 1.0, g.pad_lo, g.pad_hi, tol=1e-3, max_iter=50000,
                       check_every=16)

    with plan() as p, _design(p, prm) as d:
        h = torch.from_numpy(h0.copy()).cuda()
        d.run(h, PlaneWave(), r0, steps=2)
        d.save(path, h, fields=True)
        st = d.state_dict(h)
        m_host = np.empty(h0.shape, np.float32)
        v_host = np.empty(h0.shape, np.float32)
        t = ctypes.c_int()
        from paper_2506_15411_gb300 import _lib as L
        L.check(d.lib.cbs_design_get_state(d.handle, m_host.ctypes.data_as(ctypes.c_void_p),
                                           v_host.ctypes.data_as(ctypes.c_void_p), ctypes.byref(t)))
        a = [d.step(h, PlaneWave(), r0, warm_start=2) for _ in range(2)]
        torch.cuda.synchronize()
        h_a = h.cpu().numpy()
    assert st["t"] == 2 and t.value == 2
    assert np.array_equal(m_host, st["m"].cpu().numpy()) and np.array_equal(v_host, st["v"].cpu().numpy())
    assert float(np.abs(m_host).max()) > 0 and float(v_host.max()) > 0

    with plan() as p, _design(p, prm) as d:
        h = d.load(path)
        b = [d.step(h, PlaneWave(), r0, warm_start=2) for _ in range(2)]
        torch.cuda.synchronize()
        h_b = h.cpu().numpy()
    assert np.array_equal(h_a, h_b)
    for x, y in zip(a, b):
        assert x.objective == y.objective and x.fwd.iters == y.fwd.iters and x.adj.iters == y.adj.iters

    with plan() as p, _design(p, dataclasses.replace(prm, alpha=0.1)) as d:
        with pytest.raises(ValueError):
            d.load(path)
