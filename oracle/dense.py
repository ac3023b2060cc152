"""Dense reference solve of the discrete problem the CBS converges to.  TEST INFRASTRUCTURE
ONLY (see ``oracle/cbs_oracle.py`` for who may import it).

The vector CBS of refs. [25], [26] reaches, up to its residual, the solution of one linear
system on the periodic grid:

    A E = S,      A = C - diag(k^2),

where C is the spectral curl-curl operator: in Fourier space it multiplies the field at
wave vector p by |p|^2 I - q q^T (the symbol of curl curl = grad div - laplacian, with q = p
except that the Nyquist component of an even-length axis, whose sign is undefined, is left
out of the q q^T term so that C stays real and symmetric).  Here A
is built as an explicit matrix from 1D DFT matrices (no FFT, no Green's function) and
solved with a dense LU, on grids small enough for that (a few hundred voxels).
"""
from __future__ import annotations

import numpy as np


def dft_matrix(n: int) -> np.ndarray:
    """F[k, j] = exp(-2 pi i k j / n)."""
    k = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(k, k) / n)


def curl_curl_matrix(nx: int, ny: int, nz: int, pitch: float) -> np.ndarray:
    """Matrix of the spectral curl-curl on (3, nz, ny, nx) fields flattened C-order."""
    n = nx * ny * nz
    F = np.kron(dft_matrix(nz), np.kron(dft_matrix(ny), dft_matrix(nx)))
    Finv = F.conj().T / n
    def freqs(m):
        f = 2 * np.pi * np.fft.fftfreq(m, d=pitch)
        g = f.copy()
        if m % 2 == 0:
            g[m // 2] = 0.0
        return f, g

    (fx, gx), (fy, gy), (fz, gz) = freqs(nx), freqs(ny), freqs(nz)
    flat = lambda a: np.broadcast_to(a, (nz, ny, nx)).reshape(-1)
    P = [flat(fx[None, None, :]), flat(fy[None, :, None]), flat(fz[:, None, None])]
    Q = [flat(gx[None, None, :]), flat(gy[None, :, None]), flat(gz[:, None, None])]
    p2 = P[0] ** 2 + P[1] ** 2 + P[2] ** 2
    C = np.zeros((3 * n, 3 * n), dtype=np.complex128)
    for a in range(3):
        for b in range(3):
            sym = (p2 if a == b else 0.0) - Q[a] * Q[b]
            C[a * n:(a + 1) * n, b * n:(b + 1) * n] = Finv @ (sym[:, None] * F)
    return C


def solve(nx: int, ny: int, nz: int, pitch: float, k2: np.ndarray, S: np.ndarray) -> np.ndarray:
    """E with (C - diag(k^2)) E = S; k2 (nz, ny, nx), S (3, nz, ny, nx)."""
    n = nx * ny * nz
    A = curl_curl_matrix(nx, ny, nz, pitch)
    A[np.arange(3 * n), np.arange(3 * n)] -= np.tile(np.asarray(k2).reshape(-1), 3)
    E = np.linalg.solve(A, np.asarray(S, dtype=np.complex128).reshape(-1))
    return E.reshape((3, nz, ny, nx))
