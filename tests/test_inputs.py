"""Seeded workload generators: geometry checks against closed forms."""
from __future__ import annotations

import math

import numpy as np

from paper_2506_15411_gb300 import inputs

LAM = 1.064e-6


def test_sphere_volume_fraction_integrates_to_sphere_volume():
    n, pitch, a = 40, LAM / 8, 1.3e-6
    eps = inputs.sphere_eps(n, n, n, pitch, a, 1.5, 1.0)
    frac = (eps.astype(np.float64) - 1.0) / (1.5 ** 2 - 1.0)
    vol = frac.sum() * pitch ** 3
    assert abs(vol - 4 / 3 * math.pi * a ** 3) < 2e-3 * 4 / 3 * math.pi * a ** 3
    assert eps.dtype == np.float32 and eps.min() >= 1.0 and eps.max() <= 2.25 + 1e-6
    # symmetric under reflection about the centre
    assert np.allclose(eps, eps[::-1, ::-1, ::-1])


def test_focal_length_from_numerical_aperture():
    f = inputs.focal_length(16e-6, 0.84)
    assert math.isclose(math.sin(math.atan(8e-6 / f)), 0.84, rel_tol=1e-12)
    assert abs(f - 5.17e-6) < 0.01e-6


def test_fresnel_kinoform_phase():
    """Thickness wraps the focusing phase: (n-1) k h + k (sqrt(r^2+f^2) - f) = 0 mod 2 pi."""
    D, NA, n = 16e-6, 0.84, 1.5
    r = np.linspace(0, D / 2, 2001)
    h = inputs.fresnel_height(r, LAM, D, NA, n)
    f = inputs.focal_length(D, NA)
    k = 2 * math.pi / LAM
    phase = (n - 1) * k * h + k * (np.sqrt(r ** 2 + f ** 2) - f)
    wrapped = np.mod(phase + 1e-9, 2 * math.pi)
    assert np.all((wrapped < 1e-6) | (wrapped > 2 * math.pi - 1e-6))
    assert h.max() <= LAM / (n - 1) + 1e-15 and h.min() >= 0
    assert inputs.fresnel_height(np.array([D / 2 * 1.01]), LAM, D, NA, n)[0] == 0.0


def test_height_to_eps_subpixel_fractions():
    h = np.array([[0.0, 0.5, 1.0, 2.25]]) * 1e-7
    eps = inputs.height_to_eps(h, 6, 1e-7, 2, 1.5, 1.0)
    frac = (eps - 1.0) / 1.25
    assert np.allclose(frac[:2], 0)
    assert np.allclose(frac[2:, 0, 0], [0, 0, 0, 0])
    assert np.allclose(frac[2:, 0, 1], [0.5, 0, 0, 0])
    assert np.allclose(frac[2:, 0, 2], [1, 0, 0, 0])
    assert np.allclose(frac[2:, 0, 3], [1, 1, 0.25, 0])
    assert np.allclose(frac.sum(axis=0)[0] * 1e-7, h[0])


def test_lens_workload_layout():
    wl = inputs.fresnel_lens_workload(275, 275, 315, LAM / 16, LAM, 16e-6, 0.84, 1.5)
    assert wl.pad_lo == (16, 16, 96) and wl.eps.shape == (315, 275, 275)
    assert wl.z_base == wl.z_source + 2 and wl.r0[:2] == (137, 137)
    assert wl.r0[2] == wl.z_base + round(inputs.focal_length(16e-6, 0.84) / (LAM / 16))
    # interior spans the lens diameter (243 voxels of 66.5 nm ~ 16.2 um)
    assert (275 - 32) * LAM / 16 > 16e-6


def test_seeded_generators_are_reproducible():
    a = inputs.random_field(5, 4, 3, seed=9)
    b = inputs.random_field(5, 4, 3, seed=9)
    assert np.array_equal(a, b) and a.shape == (3, 3, 4, 5)
    e1, reg = inputs.design_slab_eps(64, 64, 48, LAM / 8, LAM, slab=(32, 32, 8), z_base=10)
    e2, _ = inputs.design_slab_eps(64, 64, 48, LAM / 8, LAM, slab=(32, 32, 8), z_base=10)
    assert np.array_equal(e1, e2)
    assert e1[reg].min() >= 1.0 and e1[reg].max() <= 2.25 + 1e-6


def test_serving_stream_is_seeded_and_poisson():
    a = inputs.serving_stream(500, seed=42, rate_hz=4.0)
    b = inputs.serving_stream(500, seed=42, rate_hz=4.0)
    assert [(q["nx"], q["structure"], q["n"], q["adjoint"], q["arrival_s"]) for q in a] == \
           [(q["nx"], q["structure"], q["n"], q["adjoint"], q["arrival_s"]) for q in b]
    gaps = np.diff([q["arrival_s"] for q in a])
    assert abs(gaps.mean() - 0.25) < 0.03 and abs(gaps.std() - 0.25) < 0.04     # exponential: mean = std
    assert {q["structure"] for q in a} == {"sphere", "lens"}
    assert all(1.3 <= q["n"] <= 1.6 for q in a)
    assert 0.4 < np.mean([q["adjoint"] for q in a]) < 0.6
    assert {(q["nx"], q["ny"], q["nz"]) for q in a} == set(inputs.SERVING_SIZES)
    for q in a[:40]:
        x, y, z = q["r0"]
        assert q["pads"][2] <= z < q["nz"] - q["pads"][2] and x == q["nx"] // 2 and y == q["ny"] // 2
    small = inputs.serving_stream(4, sizes=((32, 32, 32),), seed=1)
    e = inputs.request_eps(small[0])
    assert e.shape == (32, 32, 32) and e.dtype == np.float32 and 1.0 <= e.min() and e.max() <= 1.6 ** 2 + 1e-6


def test_balanced_serving_stream_covers_every_size_equally():
    """The measured streams draw every size n // len(sizes) times (or once more), so a short
    stream still covers all five; the draw is seeded."""
    for n in (20, 23):
        a = inputs.serving_stream(n, seed=42, balanced=True)
        b = inputs.serving_stream(n, seed=42, balanced=True)
        assert [(q["nx"], q["nz"], q["structure"], q["adjoint"]) for q in a] == \
               [(q["nx"], q["nz"], q["structure"], q["adjoint"]) for q in b]
        counts = {s: sum(1 for q in a if (q["nx"], q["ny"], q["nz"]) == s) for s in inputs.SERVING_SIZES}
        assert set(counts.values()) <= {n // 5, n // 5 + 1} and sum(counts.values()) == n
    # the order is random, not the sizes in turn
    a = inputs.serving_stream(20, seed=42, balanced=True)
    assert [q["nx"] for q in a[:5]] != [s[0] for s in inputs.SERVING_SIZES]
