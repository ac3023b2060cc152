"""FP64 CPU oracle of the vector convergent Born series (CBS) and its adjoint gradient.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
legs of ``bench.py`` may import this module.  The product path (the CUDA library and its
Python binding) never calls it, and it shares no code with that path.

What is computed, and where it comes from
-----------------------------------------
The paper (arXiv 2506.15411) solves the monochromatic Maxwell equations for the *total
electric field* of a lens under an x-polarised plane wave (Fig. 2 paragraph) with the
vector CBS of its refs. [25] (scalar CBS) and [26] (vector CBS), inside absorbing layers
of thickness [lambda, lambda, 6 lambda] (Fig. 1 benchmark paragraph).  It prints none of
the equations, so this file states them from the mathematics; every reading of a point
the paper leaves open is marked READING.

* Problem (time convention exp(-i w t), outgoing waves exp(+i k r)):
      curl curl E - k(r)^2 E = S,      k(r)^2 = k_vac^2 (eps_r(r) + i sigma(r)).
* Splitting (ref. [25]):  k(r)^2 = k0^2 + i epsilon + V(r), with
      k0^2 = (min Re k^2 + max Re k^2) / 2,   epsilon = max |k^2 - k0^2|.
* Green operator of curl curl - (k0^2 + i epsilon) on the periodic grid, in k-space
      G(p) = (I - p p^T / kt2) / (|p|^2 - kt2),   kt2 = k0^2 + i epsilon,
  with p = 2 pi fftfreq(n, pitch) per axis (the exact spectral symbol).
  READING (Nyquist): on an even-length axis the Nyquist wave number has no sign, and the
  symbol |p|^2 I - p p^T with p taken negative there is not even in p, which makes the
  discrete curl curl neither real nor symmetric.  The adjoint method needs A^T = A, so the
  p p^T term uses q = p with its Nyquist components set to 0 (|p|^2 keeps them):
      D(p) = |p|^2 I - q q^T,   G = (D - kt2)^{-1} = [I + q q^T / (|p|^2 - |q|^2 - kt2)] / (|p|^2 - kt2),
  which is the formula above wherever no component is at Nyquist (q = p).
* Preconditioned iteration (ref. [25], carried to 3 components as in ref. [26]):
      gamma = (i / epsilon) V,
      E_{k+1} = E_k - gamma [E_k - G (V E_k + S)],    E_0 = 0 (or a warm start).
  Its fixed point solves E = G (V E + S), i.e. the problem above.
* Residual: delta_k = gamma [E_k - G(V E_k + S)] = E_k - E_{k+1};
  relative residual r_k = ||delta_k|| / ||delta_0||, summed over 3 components and every
  voxel (layers included).  READING: the paper names no stopping rule.
* Adjoint and gradient of the figure of merit L = |E(r0)|^2 (Fig. 2 caption, and the
  paragraph on the figure of merit): the operator A = curl curl - k^2 is complex symmetric,
  so E_adj = A^{-1} [conj(E(r0)) delta_{r0}] is one more CBS solve with a point source of
  raw value conj(E(r0)) at voxel r0, and dL/d eps_r(r) = 2 k_vac^2 Re[E_adj(r) . E(r)].

Array layout: fields are complex128 arrays of shape (3, nz, ny, nx) (component order x, y,
z; x fastest in memory), scalar grids are (nz, ny, nx).

What pins what (tests/test_oracle_pins.py, test_mie.py): the fixed point against a dense
solve of the discrete system and the homogeneous closed form; the physics scale and time
convention against the closed-form dyadic Green function and Mie scattering; the adjoint
against reciprocity; the gradient against central differences.  Parity unpinned by the
paper: the layer profile and its strength (layer_strength, axis_profile, absorption), the
plane-wave sheet's placement (plane_wave_source) and the stopping rule are READINGS; each
is pinned only to its own stated definition (the 1e-4 round trip, the unit plane wave in a
homogeneous medium), not to a number the paper prints.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np
import scipy.fft as sfft

WORKERS = os.cpu_count() or 1
LN_1E4 = math.log(1.0e4)


@dataclass
class Grid:
    """A CBS problem grid.  ``pad_lo``/``pad_hi`` are the absorbing-layer thicknesses in
    voxels per face, ordered (x, y, z); the layers lie inside the nx*ny*nz grid."""

    nx: int
    ny: int
    nz: int
    pitch: float          # voxel pitch [m]
    lam: float            # vacuum wavelength [m]
    n_bg: float = 1.0     # background refractive index (sets the layer strength)
    pad_lo: tuple = (0, 0, 0)
    pad_hi: tuple = (0, 0, 0)
    # absorbing-layer profile (READING, see layer_strength): the round-trip amplitude a
    # normally incident plane wave keeps, the ramp exponent, and the rule where layers overlap
    round_trip: float = 1e-4
    power: float = 2.0
    corner: str = "sum"   # "sum": the axis profiles add; "max": the largest applies

    @property
    def k_vac(self) -> float:
        return 2.0 * math.pi / self.lam

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n_vox(self) -> int:
        return self.nx * self.ny * self.nz


# --------------------------------------------------------------------------------------
# Absorbing layers (Fig. 1 benchmark paragraph: thickness [lambda, lambda, 6 lambda]).
# --------------------------------------------------------------------------------------
def layer_strength(grid: Grid, thickness_vox: int) -> float:
    """Peak absorption sigma_max of one layer of the given thickness.

    READING (the paper gives no profile): k^2 gains i k_vac^2 sigma_max (t/L)^p at depth t
    into a layer of thickness L (p = grid.power, 2 by default).  For weak absorption
    Im k = k_vac sigma / (2 n_bg), so the one-way attenuation exponent is
    k_vac sigma_max L / (2 (p + 1) n_bg); sigma_max is set so that the round trip through the
    layer leaves the amplitude grid.round_trip (1e-4 by default).
    """
    L = thickness_vox * grid.pitch
    log_rt = LN_1E4 if grid.round_trip == 1e-4 else math.log(1.0 / grid.round_trip)
    return (grid.power + 1.0) * grid.n_bg * log_rt / (grid.k_vac * L)


def _ramp(t: float, p: float) -> float:
    return t * t if p == 2.0 else t ** p


def axis_profile(grid: Grid, n: int, lo: int, hi: int) -> np.ndarray:
    """sigma along one axis: zero in the interior, a ramp (t / thickness)^p in each layer.

    Voxel i < lo sits at depth t = lo - i (1..lo) into the low layer; voxel i >= n - hi at
    depth t = i - (n - hi - 1) (1..hi) into the high layer.
    """
    s = np.zeros(n)
    for i in range(n):
        if i < lo:
            s[i] = layer_strength(grid, lo) * _ramp((lo - i) / lo, grid.power)
        elif i >= n - hi:
            s[i] = layer_strength(grid, hi) * _ramp((i - (n - hi - 1)) / hi, grid.power)
    return s


def absorption(grid: Grid) -> np.ndarray:
    """sigma(r) on the grid.  READING: where layers overlap (edges, corners) the per-axis
    profiles add (grid.corner = "sum", the default) or the largest applies ("max")."""
    sx = axis_profile(grid, grid.nx, grid.pad_lo[0], grid.pad_hi[0])
    sy = axis_profile(grid, grid.ny, grid.pad_lo[1], grid.pad_hi[1])
    sz = axis_profile(grid, grid.nz, grid.pad_lo[2], grid.pad_hi[2])
    if grid.corner == "max":
        return np.maximum(np.maximum(sz[:, None, None], sy[None, :, None]), sx[None, None, :])
    if grid.corner != "sum":
        raise ValueError(f"corner rule {grid.corner!r}")
    return sz[:, None, None] + sy[None, :, None] + sx[None, None, :]


def k_squared(grid: Grid, eps_r: np.ndarray) -> np.ndarray:
    """k(r)^2 = k_vac^2 (eps_r + i sigma), complex128 (nz, ny, nx)."""
    eps_r = np.asarray(eps_r, dtype=np.float64)
    assert eps_r.shape == grid.shape
    return grid.k_vac ** 2 * (eps_r + 1j * absorption(grid))


# --------------------------------------------------------------------------------------
# Splitting and Green operator (refs. [25], [26]).
# --------------------------------------------------------------------------------------
@dataclass
class Splitting:
    k0sq: float
    epsilon: float

    @property
    def kt2(self) -> complex:
        return complex(self.k0sq, self.epsilon)


def splitting(k2: np.ndarray) -> Splitting:
    """k0^2 halfway between the extreme real parts of k^2, epsilon = max |k^2 - k0^2|
    (READING: no safety factor).  This choice of k0^2 minimises epsilon over real k0^2
    for a lossless medium."""
    re = k2.real
    k0sq = 0.5 * (float(re.min()) + float(re.max()))
    epsilon = float(np.abs(k2 - k0sq).max())
    if not epsilon > 0.0:
        raise ValueError("epsilon = 0: a lossless homogeneous grid has no convergent splitting")
    return Splitting(k0sq, epsilon)


def axis_wavenumbers(n: int, pitch: float):
    """(p, q) along one axis: p = 2 pi fftfreq(n, pitch) (NumPy convention, Nyquist bin of an
    even length negative) and q = p with the Nyquist bin set to 0."""
    p = 2.0 * np.pi * np.fft.fftfreq(n, d=pitch)
    q = p.copy()
    if n % 2 == 0:
        q[n // 2] = 0.0
    return p, q


def wavevectors(grid: Grid):
    """(p_x, p_y, p_z), (q_x, q_y, q_z), each broadcastable to (nz, ny, nx)."""
    px, qx = axis_wavenumbers(grid.nx, grid.pitch)
    py, qy = axis_wavenumbers(grid.ny, grid.pitch)
    pz, qz = axis_wavenumbers(grid.nz, grid.pitch)
    return ((px[None, None, :], py[None, :, None], pz[:, None, None]),
            (qx[None, None, :], qy[None, :, None], qz[:, None, None]))


def green_apply(grid: Grid, kt2: complex, X: np.ndarray) -> np.ndarray:
    """G X for a 3-component field X: per-component 3D FFT, multiply by the dyadic
    G = [I + q q^T / (|p|^2 - |q|^2 - kt2)] / (|p|^2 - kt2), inverse FFT.

    G is the inverse of D - kt2 I with D = |p|^2 I - q q^T, the Fourier symbol of curl curl
    (q = p away from Nyquist, where G = (I - p p^T / kt2) / (|p|^2 - kt2): transverse part
    1/(|p|^2 - kt2), longitudinal part -1/kt2)."""
    (px, py, pz), (qx, qy, qz) = wavevectors(grid)
    Xh = sfft.fftn(X, axes=(1, 2, 3), workers=WORKERS)
    p2 = px * px + py * py + pz * pz
    q2 = qx * qx + qy * qy + qz * qz
    q_dot = qx * Xh[0] + qy * Xh[1] + qz * Xh[2]
    c = q_dot / (p2 - q2 - kt2)
    denom = p2 - kt2
    Yh = np.empty_like(Xh)
    Yh[0] = (Xh[0] + qx * c) / denom
    Yh[1] = (Xh[1] + qy * c) / denom
    Yh[2] = (Xh[2] + qz * c) / denom
    return sfft.ifftn(Yh, axes=(1, 2, 3), workers=WORKERS)


# --------------------------------------------------------------------------------------
# Sources (Fig. 2 paragraph: normally incident x-polarised plane wave).
# --------------------------------------------------------------------------------------
def plane_wave_source(grid: Grid, pol=(1.0, 0.0, 0.0), z_plane: int | None = None) -> np.ndarray:
    """Current sheet launching a plane wave along +z (and -z) from voxel plane z_plane.

    READING (the paper does not say how its plane wave is injected): in a homogeneous
    background of index n_bg the 1D problem -E'' - k_b^2 E = s delta(z - z_s) is solved by
    E = exp(i k_b |z - z_s|) when s = -2 i k_b; on the grid the delta has height 1/pitch.
    So S = pol * (-2 i k_b / pitch) on every voxel of plane z_s, zero elsewhere, which makes
    pol the complex amplitude of the launched wave.  Default plane: the first interior
    plane, z_s = pad_lo[z].
    """
    if z_plane is None:
        z_plane = grid.pad_lo[2]
    kb = grid.k_vac * grid.n_bg
    S = np.zeros((3,) + grid.shape, dtype=np.complex128)
    for c in range(3):
        S[c, z_plane, :, :] = complex(pol[c]) * (-2j * kb / grid.pitch)
    return S


def point_source(grid: Grid, r0, pol) -> np.ndarray:
    """Point source: S(r0) = pol (raw discrete value at voxel r0 = (x, y, z)), else 0.
    A continuum dipole p delta(r - r0) corresponds to pol = p / pitch^3."""
    x, y, z = r0
    S = np.zeros((3,) + grid.shape, dtype=np.complex128)
    for c in range(3):
        S[c, z, y, x] = complex(pol[c])
    return S


# --------------------------------------------------------------------------------------
# The series itself.
# --------------------------------------------------------------------------------------
@dataclass
class SolveResult:
    E: np.ndarray
    iters: int
    rel_resid: float
    history: list = field(default_factory=list)   # ||delta_k|| for k = 0 .. iters-1
    split: Splitting | None = None


def cbs_solve(grid: Grid, k2: np.ndarray, S: np.ndarray, *, tol: float = 1e-6,
              max_iter: int = 100000, E0: np.ndarray | None = None,
              split: Splitting | None = None) -> SolveResult:
    """Run E_{k+1} = E_k - gamma [E_k - G(V E_k + S)] from E_0 = E0 (zero if None).

    Stops after the first iteration k with ||delta_k|| / ||delta_0|| <= tol, or after
    max_iter iterations.  tol <= 0 runs exactly max_iter iterations (the mode used for
    parity at equal iteration count).  ``split`` overrides the splitting (any k0^2 and
    epsilon >= max|k^2 - k0^2| give the same fixed point)."""
    if split is None:
        split = splitting(k2)
    kt2 = split.kt2
    V = k2 - kt2
    gamma = (1j / split.epsilon) * V
    E = np.zeros((3,) + grid.shape, dtype=np.complex128) if E0 is None else np.array(E0, dtype=np.complex128)
    hist = []
    rel = float("inf")
    it = 0
    for it in range(1, max_iter + 1):
        W = green_apply(grid, kt2, V[None] * E + S)
        delta = gamma[None] * (E - W)
        E = E - delta
        hist.append(float(np.sqrt(np.sum(np.abs(delta) ** 2))))
        rel = hist[-1] / hist[0] if hist[0] > 0 else 0.0
        if tol > 0 and rel <= tol:
            break
    return SolveResult(E=E, iters=it, rel_resid=rel, history=hist, split=split)


def forward(grid: Grid, eps_r: np.ndarray, S: np.ndarray, **kw) -> SolveResult:
    """Total field for permittivity eps_r (real, full grid) and source S."""
    return cbs_solve(grid, k_squared(grid, eps_r), S, **kw)


def adjoint_source(grid: Grid, E: np.ndarray, r0) -> np.ndarray:
    """Adjoint source of L = |E(r0)|^2: raw value conj(E(r0)) at voxel r0."""
    x, y, z = r0
    return point_source(grid, r0, np.conj(E[:, z, y, x]))


def adjoint(grid: Grid, eps_r: np.ndarray, E: np.ndarray, r0, **kw) -> SolveResult:
    """E_adj = A^{-1} [conj(E(r0)) delta_{r0}]; A is complex symmetric, so the same CBS."""
    return forward(grid, eps_r, adjoint_source(grid, E, r0), **kw)


def objective(E: np.ndarray, r0) -> float:
    """Figure of merit |E(r0)|^2 (Fig. 2 caption)."""
    x, y, z = r0
    return float(np.sum(np.abs(E[:, z, y, x]) ** 2))


def gradient(grid: Grid, E: np.ndarray, E_adj: np.ndarray) -> np.ndarray:
    """dL/d eps_r(r) = 2 k_vac^2 Re[sum_c E_adj,c(r) E_c(r)] (bilinear, not conjugated):
    dA/d eps_r(r) = -k_vac^2 at voxel r, and A^T = A."""
    return 2.0 * grid.k_vac ** 2 * np.real(np.sum(E_adj * E, axis=0))


# --------------------------------------------------------------------------------------
# Pieces the GPU path also reports, restated here for parity checks.
# --------------------------------------------------------------------------------------
def potential(grid: Grid, eps_r: np.ndarray):
    """(V, gamma, splitting) for a permittivity grid."""
    k2 = k_squared(grid, eps_r)
    sp = splitting(k2)
    V = k2 - sp.kt2
    return V, (1j / sp.epsilon) * V, sp


def one_iteration(grid: Grid, eps_r: np.ndarray, S: np.ndarray, E: np.ndarray):
    """A single update from E; returns (E_next, ||delta||)."""
    V, gamma, sp = potential(grid, eps_r)
    W = green_apply(grid, sp.kt2, V[None] * E + S)
    delta = gamma[None] * (E - W)
    return E - delta, float(np.sqrt(np.sum(np.abs(delta) ** 2)))
