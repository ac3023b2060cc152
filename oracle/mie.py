"""Mie scattering of a plane wave by a homogeneous sphere (fields, not only cross
sections).  TEST INFRASTRUCTURE ONLY.

Restated from the standard vector-spherical-harmonic solution (Bohren & Huffman, "Absorption
and Scattering of Light by Small Particles", ch. 4), time factor exp(-i w t), for the
incident field E_inc = x^ exp(i k z) in a background of wavenumber k, a sphere of radius a
and relative index m centred at the origin:

    E_inc = sum_n E_n (M1_o1n - i N1_e1n),                 E_n = i^n (2n+1) / (n(n+1))
    E_int = sum_n E_n (c_n M1_o1n - i d_n N1_e1n)          (r < a, argument m k r)
    E_sca = sum_n E_n (i a_n N3_e1n - b_n M3_o1n)          (r > a, argument k r)

with psi(x) = x j_n(x), xi(x) = x h1_n(x) and x = k a:

    a_n = [m psi(mx) psi'(x) - psi(x) psi'(mx)] / [m psi(mx) xi'(x) - xi(x) psi'(mx)]
    b_n = [psi(mx) psi'(x) - m psi(x) psi'(mx)] / [psi(mx) xi'(x) - m xi(x) psi'(mx)]
    c_n = m [psi(x) xi'(x) - xi(x) psi'(x)] / [psi(mx) xi'(x) - m xi(x) psi'(mx)]
    d_n = m [psi(x) xi'(x) - xi(x) psi'(x)] / [m psi(mx) xi'(x) - xi(x) psi'(mx)]

It is a physics check of the CBS solution for the dielectric sphere workload (the paper
validates its CBS against FDTD on a lens, Fig. 1(a); a sphere has this closed solution).
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def n_terms(x: float, m: float) -> int:
    """Series length: Wiscombe's rule on the larger of x and |m| x, plus a margin."""
    y = max(abs(x), abs(m * x))
    return int(round(y + 4.0 * y ** (1.0 / 3.0) + 2.0)) + 6


def _psi(n, z):
    return z * spherical_jn(n, z), spherical_jn(n, z) + z * spherical_jn(n, z, derivative=True)


def _xi(n, z):
    h = spherical_jn(n, z) + 1j * spherical_yn(n, z)
    dh = spherical_jn(n, z, derivative=True) + 1j * spherical_yn(n, z, derivative=True)
    return z * h, h + z * dh


def coefficients(x: float, m: float, nmax: int):
    """(a_n, b_n, c_n, d_n) for n = 1..nmax."""
    n = np.arange(1, nmax + 1)
    ps_x, dps_x = _psi(n, x)
    ps_m, dps_m = _psi(n, m * x)
    xi_x, dxi_x = _xi(n, x)
    a = (m * ps_m * dps_x - ps_x * dps_m) / (m * ps_m * dxi_x - xi_x * dps_m)
    b = (ps_m * dps_x - m * ps_x * dps_m) / (ps_m * dxi_x - m * xi_x * dps_m)
    w = ps_x * dxi_x - xi_x * dps_x
    c = m * w / (ps_m * dxi_x - m * xi_x * dps_m)
    d = m * w / (m * ps_m * dxi_x - xi_x * dps_m)
    return a, b, c, d


def angular(nmax: int, mu: np.ndarray):
    """pi_n(mu) and tau_n(mu), n = 1..nmax, by the upward recurrences
    pi_n = ((2n-1) mu pi_{n-1} - n pi_{n-2}) / (n-1), pi_0 = 0, pi_1 = 1,
    tau_n = n mu pi_n - (n+1) pi_{n-1}."""
    pi = np.zeros((nmax + 1,) + mu.shape)
    tau = np.zeros((nmax + 1,) + mu.shape)
    pi[1] = 1.0
    tau[1] = mu
    for n in range(2, nmax + 1):
        pi[n] = ((2 * n - 1) * mu * pi[n - 1] - n * pi[n - 2]) / (n - 1)
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi[1:], tau[1:]


def _harmonics(n, rho, kind, pi, tau, cphi, sphi, sth):
    """Spherical components (r, theta, phi) of M_o1n and N_e1n with radial function
    j_n (kind 1) or h1_n (kind 3); each array has shape (nmax, npoints)."""
    nn = n[:, None]
    if kind == 1:
        z = spherical_jn(nn, rho)
        dz = spherical_jn(nn, rho, derivative=True)
    else:
        z = spherical_jn(nn, rho) + 1j * spherical_yn(nn, rho)
        dz = spherical_jn(nn, rho, derivative=True) + 1j * spherical_yn(nn, rho, derivative=True)
    drz = (z + rho * dz) / rho          # [rho z_n(rho)]' / rho
    M = (np.zeros_like(z), cphi * pi * z, -sphi * tau * z)
    N = (cphi * nn * (nn + 1) * sth * pi * z / rho, cphi * tau * drz, -sphi * pi * drz)
    return M, N


def fields(k: float, a: float, m: float, points: np.ndarray, part: str = "total") -> np.ndarray:
    """Complex E (M, 3) in Cartesian components at `points` (M, 3) [m] relative to the
    sphere centre.  part: "total" (incident + scattered outside, internal inside),
    "incident" (series of the incident wave, any point), "scattered" (outside points) or
    "internal" (inside points)."""
    P = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    r = np.linalg.norm(P, axis=1)
    r = np.where(r < 1e-12 * a, 1e-12 * a, r)
    cth = np.clip(P[:, 2] / r, -1.0, 1.0)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth ** 2))
    phi = np.arctan2(P[:, 1], P[:, 0])
    cphi, sphi = np.cos(phi), np.sin(phi)
    x = k * a
    nmax = n_terms(x, m)
    n = np.arange(1, nmax + 1)
    En = (1j ** n) * (2 * n + 1) / (n * (n + 1))
    pi, tau = angular(nmax, cth)
    an, bn, cn, dn = coefficients(x, m, nmax)
    inside = r < a
    out = np.zeros((P.shape[0], 3), dtype=np.complex128)   # spherical components first

    def add(mask, rho, kind, cM, cN):
        if not np.any(mask):
            return
        M, N = _harmonics(n, rho[mask], kind, pi[:, mask], tau[:, mask],
                          cphi[mask], sphi[mask], sth[mask])
        for comp in range(3):
            out[mask, comp] += np.sum(En[:, None] * (cM[:, None] * M[comp] + cN[:, None] * N[comp]), axis=0)

    one = np.ones(nmax, dtype=np.complex128)
    if part == "incident":
        add(np.ones_like(inside), k * r, 1, one, -1j * one)
    elif part == "scattered":
        add(~inside, k * r, 3, -bn, 1j * an)
    elif part == "internal":
        add(inside, m * k * r, 1, cn, -1j * dn)
    elif part == "total":
        add(~inside, k * r, 3, -bn, 1j * an)
        add(inside, m * k * r, 1, cn, -1j * dn)
    else:
        raise ValueError(part)
    er = np.stack([sth * cphi, sth * sphi, cth], axis=1)
    et = np.stack([cth * cphi, cth * sphi, -sth], axis=1)
    ep = np.stack([-sphi, cphi, np.zeros_like(phi)], axis=1)
    E = out[:, 0:1] * er + out[:, 1:2] * et + out[:, 2:3] * ep
    if part == "total":
        # outside: the incident plane wave itself (not its truncated series)
        E[~inside, 0] += np.exp(1j * k * P[~inside, 2])
    return E


def efficiencies(x: float, m: float):
    """(Q_ext, Q_sca) from the series: Q_ext = 2/x^2 sum (2n+1) Re(a_n + b_n),
    Q_sca = 2/x^2 sum (2n+1)(|a_n|^2 + |b_n|^2)."""
    nmax = n_terms(x, m)
    n = np.arange(1, nmax + 1)
    a, b, _, _ = coefficients(x, m, nmax)
    qext = 2.0 / x ** 2 * np.sum((2 * n + 1) * np.real(a + b))
    qsca = 2.0 / x ** 2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    return float(qext), float(qsca)
