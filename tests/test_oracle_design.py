"""Pins of the design-step oracle (oracle/design.py) against external truths.

* the subpixel shape integrates to the thickness, and agrees with the workload generator's
  independent implementation;
* the surface derivative equals central differences of a linear functional of eps_r;
* the mirror average is an orthogonal projection;
* the Gaussian filter is scipy.ndimage.gaussian_filter (zero boundary, same radius), has
  variance sigma^2, conserves mass and is self-adjoint;
* the Adam update is torch.optim.Adam (float64), and a constant gradient gives steps
  alpha g / (|g| + eps);
* the chained height gradient of |E(r0)|^2 equals central differences of full solves.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch
from scipy import ndimage

from oracle import cbs_oracle as co
from oracle import dense
from oracle import design as od
from paper_2506_15411_gb300 import inputs

LAM = 1.064e-6


def test_fill_fraction_integrates_to_the_thickness():
    rng = np.random.default_rng(1)
    pitch_um, nz, zb = 0.133, 30, 4
    h = rng.uniform(0.0, (nz - zb) * pitch_um, size=(9, 7))
    f = od.fill_fraction(h, nz, pitch_um, zb)
    assert f.min() >= 0.0 and f.max() <= 1.0
    assert np.all(f[:zb] == 0.0)
    assert np.all(np.diff(f[zb:], axis=0) <= 0.0)          # filled from the base up
    np.testing.assert_allclose(f.sum(axis=0) * pitch_um, h, rtol=2e-7, atol=1e-7)
    eps = od.permittivity(h, nz, pitch_um, zb, 1.5, 1.0)
    gen = inputs.height_to_eps(h * 1e-6, nz, pitch_um * 1e-6, zb, 1.5, 1.0)
    np.testing.assert_allclose(eps, gen, atol=3e-6)


def test_surface_gradient_is_the_derivative_of_the_shape():
    rng = np.random.default_rng(2)
    pitch_um, nz, zb, nl, nb = 0.177, 24, 3, 1.54, 1.0
    u = rng.integers(0, nz - zb - 1, size=(6, 5)) + rng.uniform(0.1, 0.9, size=(6, 5))
    u[0, 0] = 0.3                                        # first voxel above the base
    h = u * pitch_um
    g = rng.standard_normal((nz, 6, 5))
    J = lambda hh: float(np.sum(g * od.permittivity(hh, nz, pitch_um, zb, nl, nb)))
    gs = od.surface_gradient(g, h, pitch_um, zb, nl, nb)
    d = 1e-3 * pitch_um
    for (y, x), _ in np.ndenumerate(h):
        hp, hm = h.copy(), h.copy()
        hp[y, x] += d
        hm[y, x] -= d
        fd = (J(hp) - J(hm)) / (2 * d)
        assert abs(fd - gs[y, x]) <= 1e-3 * abs(gs[y, x]) + 1e-9


def test_mirror_is_an_orthogonal_projection():
    rng = np.random.default_rng(3)
    for shape in [(8, 6), (7, 9)]:
        a, b = rng.standard_normal(shape), rng.standard_normal(shape)
        Pa = od.mirror(a)
        np.testing.assert_allclose(od.mirror(Pa), Pa, atol=1e-15)
        np.testing.assert_array_equal(Pa, Pa[::-1, :])
        np.testing.assert_array_equal(Pa, Pa[:, ::-1])
        assert abs(np.sum(Pa * b) - np.sum(a * od.mirror(b))) <= 1e-12 * np.abs(a).sum()


@pytest.mark.parametrize("sigma_px", [355 / 177.0, 355 / 133.0, 0.7])
def test_gaussian_filter(sigma_px):
    rng = np.random.default_rng(4)
    a = rng.standard_normal((40, 33))
    R = int(np.ceil(4 * sigma_px))
    ref = ndimage.gaussian_filter(a, sigma_px, mode="constant", cval=0.0, radius=R)
    np.testing.assert_allclose(od.smooth(a, sigma_px), ref, atol=1e-12)
    w = od.gaussian_weights(sigma_px)
    k = np.arange(-R, R + 1)
    assert abs(w.sum() - 1.0) <= 1e-15
    if sigma_px >= 1.5:
        # variance sigma^2, short of it by the second moment of the tails beyond ceil(4 sigma)
        # (up to ~3e-4 of it)
        assert abs(np.sum(k ** 2 * w) - sigma_px ** 2) <= 1e-3 * sigma_px ** 2
    d = np.zeros((40, 33))
    d[20, 16] = 1.0
    assert abs(od.smooth(d, sigma_px).sum() - 1.0) <= 1e-12
    b = rng.standard_normal((40, 33))
    assert abs(np.sum(od.smooth(a, sigma_px) * b) - np.sum(a * od.smooth(b, sigma_px))) <= 1e-11
    np.testing.assert_array_equal(od.smooth(a, 0.0), a)


def test_adam_matches_torch_and_constant_gradient_steps():
    rng = np.random.default_rng(5)
    prm = od.DesignParams(z_base=0, n_lens=1.5, aperture_um=1e9, h_max_um=1e9, alpha=0.3)
    h = rng.uniform(1.0, 2.0, size=(5, 4))
    mask = np.ones(h.shape, dtype=bool)
    st = od.AdamState.zeros(h.shape)
    p = torch.nn.Parameter(torch.from_numpy(h.copy()))
    opt = torch.optim.Adam([p], lr=0.3, betas=(0.9, 0.999), eps=1e-6)
    for _ in range(6):
        g = rng.standard_normal(h.shape)
        h = od.adam_update(h, g, st, prm, mask)
        p.grad = torch.from_numpy(g.copy())
        opt.step()
        np.testing.assert_allclose(h, p.detach().numpy(), rtol=0, atol=1e-12)
    # constant gradient: bias-corrected moments are g and g^2 at every step
    st = od.AdamState.zeros((3,))
    g = np.array([2.0, -0.5, 1e-7])
    x = np.zeros(3) + 10.0
    for _ in range(4):
        xn = od.adam_update(x, g, st, prm, np.ones(3, dtype=bool))
        np.testing.assert_allclose(x - xn, 0.3 * g / (np.abs(g) + 1e-6), rtol=1e-9)
        x = xn


def test_constraints_box_and_aperture():
    prm = od.DesignParams(z_base=0, n_lens=1.5, aperture_um=1.0, h_max_um=1.0, alpha=0.3)
    mask = od.aperture(9, 9, 0.2, prm.aperture_um)
    assert mask[4, 4] and not mask[0, 0] and mask.sum() == 21     # |(i, j)| <= 2.5 pixels
    st = od.AdamState.zeros((9, 9))
    h = np.full((9, 9), 0.95)
    h[4, 3] = 0.1
    g = np.ones((9, 9))
    g[4, 4] = -1.0
    hn = od.adam_update(h, g, st, prm, mask)
    assert np.all(hn[~mask] == 0.0)
    assert hn[4, 4] == 1.0 and hn[4, 3] == 0.0           # clamped at h_max and at 0
    assert np.all(st.m[~mask] == 0.0)


@pytest.mark.parametrize("sigma_um,mirror", [(0.0, False), (0.355, True)])
def test_height_gradient_matches_central_differences(sigma_um, mirror):
    """d|E(r0)|^2/dh through smoothing, symmetry, subpixel shape and an adjoint solve, against
    central differences of L.  Both sides use the dense solve of the discrete system (no
    series), in a lossy medium k^2 = k_vac^2 (eps_r + 0.3 i) without absorbing layers."""
    g = co.Grid(8, 8, 10, LAM / 6, LAM, 1.0)
    p_um = g.pitch * 1e6
    prm = od.DesignParams(z_base=2, n_lens=1.5, aperture_um=10.0, h_max_um=2.0, sigma_um=sigma_um, mirror=mirror)
    rng = np.random.default_rng(9)
    h = rng.uniform(0.2, 1.0, size=(g.ny, g.nx))
    S = co.plane_wave_source(g, z_plane=1)
    r0 = (4, 3, 8)
    n = g.n_vox
    C = dense.curl_curl_matrix(g.nx, g.ny, g.nz, g.pitch)

    def solve(k2, src):
        A = C.copy()
        A[np.arange(3 * n), np.arange(3 * n)] -= np.tile(k2.reshape(-1), 3)
        return np.linalg.solve(A, src.reshape(-1)).reshape((3,) + g.shape)

    def fields(hh):
        he = od.effective_height(hh, p_um, prm)
        eps = od.permittivity(he, g.nz, p_um, prm.z_base, prm.n_lens, g.n_bg)
        k2 = g.k_vac ** 2 * (eps + 0.3j)
        return solve(k2, S), k2, he

    E, k2, he = fields(h)
    E_adj = solve(k2, co.adjoint_source(g, E, r0))
    gh = od.height_gradient(co.gradient(g, E, E_adj), he, p_um, prm, g.n_bg)
    d = 1e-5
    u0 = np.floor(od.surface_coordinate(he, p_um))
    checked = 0
    for (y, x) in [(3, 4), (1, 2), (6, 5), (0, 7)]:
        vals = []
        for s in (+1, -1):
            hh = h.copy()
            hh[y, x] += s * d
            Es, _, hes = fields(hh)
            # a difference across a voxel face is not a derivative: skip that pixel
            if not np.array_equal(np.floor(od.surface_coordinate(hes, p_um)), u0):
                break
            vals.append(co.objective(Es, r0))
        if len(vals) < 2:
            continue
        fd = (vals[0] - vals[1]) / (2 * d)
        assert abs(fd - gh[y, x]) <= 1e-5 * abs(fd) + 1e-8 * np.abs(gh).max(), (y, x, fd, gh[y, x])
        checked += 1
    assert checked >= 3
