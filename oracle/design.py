"""FP64 oracle of one inverse-design step on the lens thickness map (Section 3, Fig. 2(a)).

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the benchmark's CPU
baseline, never by the product path.

Design variables: the thickness map h(x, y) in micrometres over the lateral grid.  A step
    h_eff = G_sigma[M h]                        mirror symmetry M, optional Gaussian G_sigma
    eps_r = eps_bg + f(h_eff) (eps_lens - eps_bg)   shape S(r) = Theta(h - z), subpixel along z
    E, E_adj, dL/d eps_r                        forward / adjoint CBS (cbs_oracle)
    dL/dh = M G_sigma [dL/dh_eff]                chain rule (M and G_sigma are symmetric)
    h <- Adam(h, -dL/dh)                         ascent on L = |E(r0)|^2
Readings where the paper is silent:
  * f in voxel k = z - z_base >= 0 is clamp(u - k, 0, 1), u = h / pitch (the same subpixel
    rule as the workload generator); below the base f = 0.  dL/dh_eff(x, y) is the
    derivative from above: (eps_lens - eps_bg) / pitch times dL/d eps_r at the one voxel
    with 0 <= u - k < 1.
  * M averages h over the four mirror images (x, y) -> (+-x, +-y) about the grid centre.
  * G_sigma: separable, weights exp(-k^2 / 2 s^2), |k| <= ceil(4 s), s = sigma / pitch,
    normalised to sum 1; zero outside the grid.
  * Adam (Kingma & Ba, Algorithm 1) on the loss -L with h and alpha in micrometres,
    bias-corrected moments; afterwards h is clamped to [0, h_max] and set to 0 outside
    the aperture r <= D/2 (there the moments are not updated).
Parity unpinned by the paper: these readings (units, subpixel rule, mirror average, filter
radius, constraints) are pinned to their own definitions (scipy's Gaussian filter, torch's
Adam, central differences of dense solves; tests/test_oracle_design.py), not to a number the
paper prints.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import cbs_oracle as co


@dataclass
class DesignParams:
    z_base: int                 # voxel index of the lens base plane
    n_lens: float
    aperture_um: float          # diameter D of the design region
    h_max_um: float
    sigma_um: float = 0.0       # Gaussian smoothing std; 0: off
    mirror: bool = True
    alpha: float = 0.3          # Adam step (micrometres), Section 3
    beta1: float = 0.9
    beta2: float = 0.999
    adam_eps: float = 1e-6


@dataclass
class AdamState:
    m: np.ndarray
    v: np.ndarray
    t: int = 0

    @staticmethod
    def zeros(shape):
        return AdamState(np.zeros(shape), np.zeros(shape), 0)


def surface_coordinate(h_um: np.ndarray, pitch_um: float) -> np.ndarray:
    """u = h / pitch: the height in voxels above the base plane."""
    return np.asarray(h_um, dtype=np.float64) / pitch_um


def fill_fraction(h_um: np.ndarray, nz: int, pitch_um: float, z_base: int) -> np.ndarray:
    """f(z, y, x) = clamp(u - (z - z_base), 0, 1) for z >= z_base, else 0."""
    u = surface_coordinate(h_um, pitch_um)
    f = np.zeros((nz,) + u.shape)
    for z in range(max(z_base, 0), nz):
        f[z] = np.clip(u - (z - z_base), 0.0, 1.0)
    return f


def permittivity(h_um, nz, pitch_um, z_base, n_lens, n_bg):
    """eps_r of the shape function S(r) = Theta(h(r_perp) - z) with subpixel filling."""
    eb, el = n_bg ** 2, n_lens ** 2
    return eb + fill_fraction(h_um, nz, pitch_um, z_base) * (el - eb)


def surface_gradient(grad_eps: np.ndarray, h_um, pitch_um, z_base, n_lens, n_bg) -> np.ndarray:
    """dL/dh(x, y) = sum_z dL/d eps_r(z, y, x) d eps_r / dh: only the voxel with
    0 <= u - (z - z_base) < 1 depends on h, with slope (eps_lens - eps_bg) / pitch."""
    nz = grad_eps.shape[0]
    u = surface_coordinate(h_um, pitch_um)
    k = np.floor(u).astype(np.int64)
    out = np.zeros(u.shape)
    slope = (n_lens ** 2 - n_bg ** 2) / pitch_um
    for (y, x), kk in np.ndenumerate(k):
        z = z_base + kk
        if kk >= 0 and z < nz:
            out[y, x] = slope * grad_eps[z, y, x]
    return out


def mirror(h: np.ndarray) -> np.ndarray:
    """Average over (x, y) -> (+-x, +-y) about the grid centre, summed pairwise (x pairs, then
    y pairs) so that the result is exactly symmetric in floating point."""
    s = h + h[:, ::-1]
    return 0.25 * (s + s[::-1, :])


def gaussian_weights(sigma_px: float) -> np.ndarray:
    R = int(math.ceil(4.0 * sigma_px))
    k = np.arange(-R, R + 1, dtype=np.float64)
    w = np.exp(-k ** 2 / (2.0 * sigma_px ** 2))
    return w / w.sum()


def _filter_axis(a: np.ndarray, w: np.ndarray, axis: int) -> np.ndarray:
    R = (len(w) - 1) // 2
    a = np.moveaxis(a, axis, -1)
    n = a.shape[-1]
    out = np.zeros_like(a, dtype=np.float64)
    for j, wk in enumerate(w):
        k = j - R                       # out[i] += w_k a[i + k]
        lo, hi = max(0, -k), min(n, n - k)
        if lo < hi:
            out[..., lo:hi] += wk * a[..., lo + k:hi + k]
    return np.moveaxis(out, -1, axis)


def smooth(h: np.ndarray, sigma_px: float) -> np.ndarray:
    """Separable Gaussian filter, zero outside the grid; identity for sigma_px <= 0."""
    if sigma_px <= 0:
        return np.array(h, dtype=np.float64)
    w = gaussian_weights(sigma_px)
    return _filter_axis(_filter_axis(np.asarray(h, dtype=np.float64), w, 1), w, 0)


def aperture(nx: int, ny: int, pitch_um: float, D_um: float) -> np.ndarray:
    """Pixels whose centre lies within r <= D/2 of the grid centre."""
    x = (np.arange(nx) - (nx - 1) / 2.0) * pitch_um
    y = (np.arange(ny) - (ny - 1) / 2.0) * pitch_um
    return (x[None, :] ** 2 + y[:, None] ** 2) <= (D_um / 2.0) ** 2


def effective_height(h_um, pitch_um, prm: DesignParams) -> np.ndarray:
    hm = mirror(h_um) if prm.mirror else np.asarray(h_um, dtype=np.float64)
    return smooth(hm, prm.sigma_um / pitch_um)


def height_gradient(grad_eps, h_eff, pitch_um, prm: DesignParams, n_bg: float) -> np.ndarray:
    """dL/dh from dL/d eps_r: the surface derivative, then the adjoints of G_sigma and M."""
    gs = surface_gradient(grad_eps, h_eff, pitch_um, prm.z_base, prm.n_lens, n_bg)
    gs = smooth(gs, prm.sigma_um / pitch_um)
    return mirror(gs) if prm.mirror else gs


def adam_update(h, grad_loss, st: AdamState, prm: DesignParams, mask):
    """One Adam step on the loss gradient, then the box and aperture constraints.
    Returns the new h; st is updated in place."""
    st.t += 1
    g = np.where(mask, grad_loss, 0.0)
    m = np.where(mask, prm.beta1 * st.m + (1 - prm.beta1) * g, st.m)
    v = np.where(mask, prm.beta2 * st.v + (1 - prm.beta2) * g ** 2, st.v)
    st.m, st.v = m, v
    mh = m / (1 - prm.beta1 ** st.t)
    vh = v / (1 - prm.beta2 ** st.t)
    hn = h - prm.alpha * mh / (np.sqrt(vh) + prm.adam_eps)
    hn = np.clip(hn, 0.0, prm.h_max_um)
    return np.where(mask, hn, 0.0)


@dataclass
class StepResult:
    h: np.ndarray
    objective: float
    grad_h: np.ndarray            # dL/dh
    h_eff: np.ndarray
    E: np.ndarray
    E_adj: np.ndarray
    fwd: co.SolveResult | None = None
    adj: co.SolveResult | None = None
    extra: dict = field(default_factory=dict)


def design_step(grid: co.Grid, h_um, st: AdamState, prm: DesignParams, S, r0, **solve_kw) -> StepResult:
    """Forward, adjoint and one Adam ascent step of |E(r0)|^2 on h (module docstring)."""
    p_um = grid.pitch * 1e6
    h_eff = effective_height(h_um, p_um, prm)
    eps = permittivity(h_eff, grid.nz, p_um, prm.z_base, prm.n_lens, grid.n_bg)
    fwd = co.forward(grid, eps, S, **solve_kw)
    adj = co.adjoint(grid, eps, fwd.E, r0, **solve_kw)
    g_eps = co.gradient(grid, fwd.E, adj.E)
    gh = height_gradient(g_eps, h_eff, p_um, prm, grid.n_bg)
    mask = aperture(grid.nx, grid.ny, p_um, prm.aperture_um)
    hn = adam_update(np.asarray(h_um, dtype=np.float64), -gh, st, prm, mask)
    return StepResult(hn, co.objective(fwd.E, r0), gh, h_eff, fwd.E, adj.E, fwd, adj)
