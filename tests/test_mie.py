"""Mie series pins (closed forms and boundary conditions) and a physics check of the CBS
oracle against Mie scattering by a dielectric sphere."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import cbs_oracle as co
from oracle import mie
from paper_2506_15411_gb300 import inputs


def test_incident_series_reproduces_plane_wave():
    k, a = 2 * np.pi, 0.7
    rng = np.random.default_rng(0)
    P = rng.uniform(-0.9, 0.9, (60, 3))
    Ei = mie.fields(k, a, 1.5, P, part="incident")
    ex = np.zeros_like(Ei)
    ex[:, 0] = np.exp(1j * k * P[:, 2])
    assert np.max(np.abs(Ei - ex)) < 1e-6


def test_small_sphere_internal_field_is_electrostatic():
    """x -> 0: uniform internal field 3 / (m^2 + 2) along the incident polarisation."""
    k, a, m = 2 * np.pi, 1e-4, 1.5
    rng = np.random.default_rng(1)
    P = rng.uniform(-0.5, 0.5, (20, 3)) * a
    E = mie.fields(k, a, m, P, part="internal")
    assert np.allclose(E[:, 0], 3 / (m * m + 2), rtol=1e-3)
    assert np.max(np.abs(E[:, 1:])) < 1e-3


def test_boundary_conditions_on_the_sphere():
    """Tangential E continuous and m^2 E_r(in) = E_r(out) at r = a."""
    k, a, m = 2 * np.pi, 0.7, 1.5
    rng = np.random.default_rng(2)
    th, ph = rng.uniform(0.1, 3.0, 30), rng.uniform(0, 2 * np.pi, 30)
    u = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    Ein = mie.fields(k, a, m, u * a * (1 - 1e-10), "internal")
    Eout = mie.fields(k, a, m, u * a * (1 + 1e-10), "total")
    tan = lambda E: E - np.sum(E * u, 1)[:, None] * u
    assert np.max(np.abs(tan(Ein) - tan(Eout))) < 1e-7
    assert np.max(np.abs(m * m * np.sum(Ein * u, 1) - np.sum(Eout * u, 1))) < 1e-7


def test_rayleigh_and_large_sphere_efficiencies():
    x, m = 0.05, 1.5
    qext, qsca = mie.efficiencies(x, m)
    ray = 8 / 3 * x ** 4 * abs((m * m - 1) / (m * m + 2)) ** 2
    assert abs(qsca - ray) < 1e-3 * ray and abs(qext - qsca) < 1e-12   # lossless
    qext_big, _ = mie.efficiencies(200.0, m)
    assert abs(qext_big - 2.0) < 0.1                                     # extinction paradox


@pytest.mark.slow
def test_cbs_scattered_field_matches_mie():
    """Scattered-field form of the sphere problem: S = k_vac^2 (eps_r - 1) E_inc with the
    exact incident plane wave, absorbing layers 1.75 wavelengths thick.  The CBS scattered
    field agrees with the Mie series to the accuracy of the lambda/8 volume-averaged sphere
    (measured about 7 % outside, 4 % inside; a flipped time convention or a missing vector
    term is off by order one)."""
    lam, n, ppl, pad, a, m = 1.0, 48, 8, 14, 0.6, 1.5
    g = co.Grid(n, n, n, lam / ppl, lam, 1.0, (pad,) * 3, (pad,) * 3)
    eps = inputs.sphere_eps(n, n, n, g.pitch, a, m, 1.0).astype(np.float64)
    x = inputs.centred_coords(n, g.pitch)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    Einc = np.zeros((3,) + g.shape, complex)
    Einc[0] = np.exp(1j * g.k_vac * Z)
    res = co.forward(g, eps, g.k_vac ** 2 * (eps - 1.0)[None] * Einc, tol=1e-6, max_iter=50000)
    P = np.stack([X, Y, Z], -1).reshape(-1, 3)
    R = np.linalg.norm(P, axis=1)
    interior = np.all(np.abs(P) < (n / 2 - pad - 1) * g.pitch, axis=1)
    Es = res.E.reshape(3, -1).T
    out = (R >= a + 2 * g.pitch) & interior
    Em = mie.fields(g.k_vac, a, m, P[out], "scattered")
    assert np.linalg.norm(Es[out] - Em) / np.linalg.norm(Em) < 0.10
    ins = R < a - 2 * g.pitch
    Em = mie.fields(g.k_vac, a, m, P[ins], "internal")
    Em[:, 0] -= np.exp(1j * g.k_vac * P[ins, 2])
    assert np.linalg.norm(Es[ins] - Em) / np.linalg.norm(Em) < 0.08
