"""Closed-form free-space dyadic Green's function.  TEST INFRASTRUCTURE ONLY.

For curl curl E - k^2 E = p delta(r - r0) in a homogeneous lossless medium (time factor
exp(-i w t)), the outgoing solution is E(r) = G(R) p with R = r - r0 and

    G(R) = g(R) [ (1 + i/(kR) - 1/(kR)^2) I + (-1 - 3i/(kR) + 3/(kR)^2) R^ R^T ],
    g(R) = exp(i k R) / (4 pi R),

i.e. G = (I + grad grad / k^2) g, the textbook electric dyadic Green's function.  It pins
the scale, the sign of the time convention and the vector (longitudinal + transverse)
structure of the discrete solver against physics that the paper relies on (refs. [25],
[26] and the problem paragraph of Fig. 2).
"""
from __future__ import annotations

import numpy as np


def dyadic_green(k: float, R: np.ndarray) -> np.ndarray:
    """G(R) for separation vectors R of shape (..., 3); returns (..., 3, 3) complex."""
    R = np.asarray(R, dtype=np.float64)
    r = np.linalg.norm(R, axis=-1)
    u = R / r[..., None]
    kr = k * r
    g = np.exp(1j * kr) / (4 * np.pi * r)
    a = 1 + 1j / kr - 1 / kr ** 2
    b = -1 - 3j / kr + 3 / kr ** 2
    eye = np.eye(3)
    return g[..., None, None] * (a[..., None, None] * eye + b[..., None, None] * u[..., :, None] * u[..., None, :])


def dipole_field(k: float, r0, p, points) -> np.ndarray:
    """E at `points` (M, 3) from dipole moment p at r0: G(points - r0) p, shape (M, 3)."""
    G = dyadic_green(k, np.asarray(points, dtype=np.float64) - np.asarray(r0, dtype=np.float64))
    return np.einsum("mij,j->mi", G, np.asarray(p, dtype=np.complex128))
