"""Seeded synthetic inputs for the CBS solver: permittivity grids and random fields.

This module holds geometry only (which voxel is lens, sphere or background, and by what
volume fraction); none of the solver's arithmetic lives here.  Both the CUDA path and the
CPU oracle receive the arrays it produces.

Workloads follow the paper's problem statement: a dielectric sphere, a Fresnel lens of
diameter D and numerical aperture NA at wavelength lambda (Fig. 1 benchmark paragraph),
with the focal length from sin^-1(NA) = tan^-1(D / 2 f_eff) (Fig. 2 caption), and a
continuous design slab around a Fresnel profile.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_STRUCTURE = 0
SEED_NOISE = 1234


def centred_coords(n: int, pitch: float) -> np.ndarray:
    """Voxel-centre coordinates symmetric about the grid centre: (i - (n-1)/2) * pitch."""
    return (np.arange(n) - (n - 1) / 2.0) * pitch


def sphere_eps(nx, ny, nz, pitch, radius, n_sphere, n_bg=1.0, centre=None, supersample=8):
    """Relative permittivity of a sphere, volume-fraction averaged over each voxel.

    Voxels whose corners are all inside (outside) get eps_sphere (eps_bg); the others are
    sampled on a supersample^3 sub-grid (isotropic volume-fraction average).
    Returns float32 (nz, ny, nx)."""
    cx, cy, cz = (0.0, 0.0, 0.0) if centre is None else centre
    x = centred_coords(nx, pitch) - cx
    y = centred_coords(ny, pitch) - cy
    z = centred_coords(nz, pitch) - cz
    e_in, e_out = n_sphere ** 2, n_bg ** 2
    half_diag = 0.5 * math.sqrt(3.0) * pitch
    out = np.empty((nz, ny, nx), dtype=np.float32)
    sub = (np.arange(supersample) + 0.5) / supersample - 0.5
    for k in range(nz):
        r = np.sqrt(z[k] ** 2 + y[:, None] ** 2 + x[None, :] ** 2)
        frac = np.where(r + half_diag <= radius, 1.0, 0.0)
        edge = np.abs(r - radius) < half_diag
        jj, ii = np.nonzero(edge)
        if len(jj):
            sx = x[ii][:, None, None, None] + sub[None, None, None, :] * pitch
            sy = y[jj][:, None, None, None] + sub[None, None, :, None] * pitch
            sz = z[k] + sub[None, :, None, None] * pitch
            inside = (sx ** 2 + sy ** 2 + sz ** 2) <= radius ** 2
            frac[jj, ii] = inside.reshape(len(jj), -1).mean(axis=1)
        out[k] = (e_out + frac * (e_in - e_out)).astype(np.float32)
    return out


def focal_length(D: float, NA: float) -> float:
    """f_eff with sin^-1(NA) = tan^-1(D / (2 f_eff))."""
    return (D / 2.0) / math.tan(math.asin(NA))


def fresnel_height(r: np.ndarray, lam: float, D: float, NA: float, n_lens: float, n_bg: float = 1.0):
    """Kinoform thickness h(r): one wrapped 2 pi phase ramp per zone, maximum
    lam / (n_lens - n_bg), zero outside r > D/2, focusing at f_eff."""
    f = focal_length(D, NA)
    hmax = lam / (n_lens - n_bg)
    path = (np.sqrt(r ** 2 + f ** 2) - f) / lam
    h = hmax * (1.0 - (path - np.floor(path)))
    return np.where(r <= D / 2.0, h, 0.0)


def height_to_eps(h: np.ndarray, nz: int, pitch: float, z_base: int, n_lens: float, n_bg: float = 1.0):
    """Shape S(r) = Theta(h(r_perp) - (z - z_base)) with subpixel averaging along z: voxel
    k >= z_base is filled by the fraction clamp((h - (k - z_base) pitch) / pitch, 0, 1).
    h is (ny, nx); returns float32 (nz, ny, nx)."""
    k = np.arange(nz)[:, None, None] - z_base
    frac = np.clip((h[None, :, :] - k * pitch) / pitch, 0.0, 1.0)
    frac = np.where(k >= 0, frac, 0.0)
    e_in, e_out = n_lens ** 2, n_bg ** 2
    return (e_out + frac * (e_in - e_out)).astype(np.float32)


@dataclass
class LensWorkload:
    nx: int
    ny: int
    nz: int
    pitch: float
    lam: float
    pad_lo: tuple
    pad_hi: tuple
    eps: np.ndarray          # float32 (nz, ny, nx)
    z_source: int            # plane-wave sheet
    z_base: int              # lens base plane (voxel index)
    r0: tuple                # focal voxel (x, y, z)
    D: float
    NA: float
    n_lens: float
    n_bg: float


def fresnel_lens_workload(nx, ny, nz, pitch, lam, D, NA, n_lens, n_bg=1.0,
                          pad_lo=None, pad_hi=None) -> LensWorkload:
    """Fresnel lens in the grid centre; x-polarised plane wave launched from the first
    interior z plane; lens base two voxels above it; focus f_eff above the base."""
    if pad_lo is None:
        p = int(round(lam / pitch))
        pad_lo = (p, p, 6 * p)
    if pad_hi is None:
        pad_hi = pad_lo
    x = centred_coords(nx, pitch)
    y = centred_coords(ny, pitch)
    r = np.sqrt(x[None, :] ** 2 + y[:, None] ** 2)
    h = fresnel_height(r, lam, D, NA, n_lens, n_bg)
    z_source = pad_lo[2]
    z_base = z_source + 2
    eps = height_to_eps(h, nz, pitch, z_base, n_lens, n_bg)
    zf = z_base + int(round(focal_length(D, NA) / pitch))
    if zf >= nz - pad_hi[2]:
        raise ValueError("focal point falls outside the interior")
    r0 = (nx // 2, ny // 2, zf)
    return LensWorkload(nx, ny, nz, pitch, lam, tuple(pad_lo), tuple(pad_hi), eps,
                        z_source, z_base, r0, D, NA, n_lens, n_bg)


def design_slab_eps(nx, ny, nz, pitch, lam, slab=(192, 192, 48), D=None, NA=0.84,
                    n_lens=1.5, n_bg=1.0, z_base=None, noise=0.1, seed=SEED_NOISE):
    """Continuous-permittivity design slab: a Fresnel profile inside a (sx, sy, sz) slab
    centred laterally, plus seeded U(-noise, noise), clipped to [n_bg^2, n_lens^2]."""
    sx, sy, sz = slab
    if D is None:
        D = sx * pitch
    x = centred_coords(nx, pitch)
    y = centred_coords(ny, pitch)
    r = np.sqrt(x[None, :] ** 2 + y[:, None] ** 2)
    h = fresnel_height(r, lam, D, NA, n_lens, n_bg)
    eps = height_to_eps(h, nz, pitch, z_base, n_lens, n_bg).astype(np.float64)
    rng = np.random.default_rng(seed)
    x0, y0 = (nx - sx) // 2, (ny - sy) // 2
    region = (slice(z_base, z_base + sz), slice(y0, y0 + sy), slice(x0, x0 + sx))
    eps[region] += rng.uniform(-noise, noise, size=(sz, sy, sx))
    eps[region] = np.clip(eps[region], n_bg ** 2, n_lens ** 2)
    return eps.astype(np.float32), region


def random_field(nx, ny, nz, seed=SEED_NOISE, scale=1.0) -> np.ndarray:
    """Seeded complex128 (3, nz, ny, nx) field with N(0, scale^2) real and imaginary parts."""
    rng = np.random.default_rng(seed)
    shape = (3, nz, ny, nx)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def random_eps(nx, ny, nz, lo=1.0, hi=2.25, seed=SEED_NOISE) -> np.ndarray:
    """Seeded uniform random permittivity, float32 (nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(nz, ny, nx)).astype(np.float32)


# ------------------------------------------------------------------ serving request streams
def parse_size(s: str) -> tuple:
    """'64' -> (64, 64, 64); '192x192x128' -> (192, 192, 128)."""
    parts = [int(v) for v in str(s).lower().split("x")]
    return tuple(parts * 3) if len(parts) == 1 else tuple(parts)


SERVING_SIZES = ((64, 64, 64), (128, 128, 128), (192, 192, 128), (256, 256, 192), (384, 384, 256))
SEED_STREAM = 42


def serving_stream(n: int, sizes=SERVING_SIZES, seed: int = SEED_STREAM, ppl: int = 8, lam: float = 1.064e-6,
                   p_adjoint: float = 0.5, rate_hz: float | None = None, balanced: bool = False) -> list:
    """Seeded request mix: grid uniform over `sizes` at pitch lam / ppl with one-wavelength
    absorbing layers on every face, a centred sphere (radius 1.5 um or 0.3 of the interior,
    the smaller) or a Fresnel lens (D = 0.7 of the lateral interior), equal odds, of index
    U[1.3, 1.6], an x-polarised plane wave, forward only or forward + adjoint (p_adjoint).
    balanced: every size equally often (n // len(sizes) or one more), in random order, so that
    a short stream still covers every size.  Each request is a dict; arrivals (Poisson,
    rate_hz) are added when rate_hz is given."""
    rng = np.random.default_rng(seed)
    pitch = lam / ppl
    order = rng.permutation(np.resize(np.arange(len(sizes)), n)) if balanced else None
    out = []
    for i in range(n):
        nx, ny, nz = sizes[int(order[i] if balanced else rng.integers(len(sizes)))]
        kind = "sphere" if rng.random() < 0.5 else "lens"
        n_idx = float(rng.uniform(1.3, 1.6))
        adj = bool(rng.random() < p_adjoint)
        pads = (ppl, ppl, ppl)
        rq = {"index": i, "nx": nx, "ny": ny, "nz": nz, "pitch": pitch, "lam": lam, "pads": pads,
              "structure": kind, "n": n_idx, "adjoint": adj, "pol": (1.0, 0.0, 0.0)}
        rq["r0"] = request_focus(rq)
        out.append(rq)
    if rate_hz:
        assign_arrivals(out, rate_hz, seed)
    return out


def assign_arrivals(reqs: list, rate_hz: float, seed: int = SEED_STREAM):
    """Poisson arrivals: exponential gaps of mean 1 / rate_hz (seed + 1), starting at 0."""
    rng = np.random.default_rng(seed + 1)
    t = 0.0
    for k, rq in enumerate(reqs):
        if k:
            t += float(rng.exponential(1.0 / rate_hz))
        rq["arrival_s"] = t


def _sphere_radius(rq) -> float:
    """1.5 um (the sphere of the 64^3 workload), or 0.3 of the interior if that is smaller:
    a larger high-index sphere is a resonator the series needs 1e5+ iterations for."""
    inner = min(rq["nx"], rq["ny"], rq["nz"]) - 2 * max(rq["pads"])
    return min(1.5e-6, 0.3 * inner * rq["pitch"])


def _lens_diameter(rq) -> float:
    return 0.7 * (min(rq["nx"], rq["ny"]) - 2 * max(rq["pads"][:2])) * rq["pitch"]


def request_focus(rq) -> tuple:
    """Objective voxel: behind the sphere's far side, or at the lens focus (clipped into the
    interior)."""
    nx, ny, nz, p = rq["nx"], rq["ny"], rq["nz"], rq["pitch"]
    z_hi = nz - rq["pads"][2] - 1
    if rq["structure"] == "sphere":
        z = int(round((nz - 1) / 2 + _sphere_radius(rq) / p)) + 2
    else:
        z = rq["pads"][2] + 2 + int(round(focal_length(_lens_diameter(rq), 0.84) / p))
    return (nx // 2, ny // 2, min(z, z_hi))


def request_eps(rq) -> np.ndarray:
    """Permittivity of a request from serving_stream (float32 (nz, ny, nx))."""
    nx, ny, nz, p = rq["nx"], rq["ny"], rq["nz"], rq["pitch"]
    if rq["structure"] == "sphere":
        return sphere_eps(nx, ny, nz, p, _sphere_radius(rq), rq["n"])
    x = centred_coords(nx, p)
    y = centred_coords(ny, p)
    r = np.sqrt(x[None, :] ** 2 + y[:, None] ** 2)
    h = fresnel_height(r, rq["lam"], _lens_diameter(rq), 0.84, rq["n"])
    return height_to_eps(h, nz, p, rq["pads"][2] + 2, rq["n"])
