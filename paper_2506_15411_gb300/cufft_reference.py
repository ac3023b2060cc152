"""The CBS iteration written with cuFFT (torch.fft) and element-wise torch operations, for
timing and cross-checking beside the fused kernels.  The solver never uses it.

One iteration here is what a straightforward GPU implementation does -- 3D FFTs of the three
components (cuFFT), the dyadic Green multiply, inverse FFTs, the update and the residual as
separate element-wise kernels:

    W = FFT(V E + S);  W <- G(p) W;  W = IFFT(W);  delta = gamma (E - W);  E -= delta

with G(p) = [I + q q^T / (|p|^2 - |q|^2 - kt2)] / (|p|^2 - kt2), q = p with Nyquist
components set to zero, kt2 = k0^2 + i epsilon, gamma = (i / epsilon) V, V = k^2 - kt2 and
k^2 = k_vac^2 (eps_r + i sigma) with the quadratic absorbing layers (peak sigma
3 n_bg ln(1e4) / (k_vac L) on a layer of L, overlapping layers adding) -- the same readings
as the CUDA path, restated here in torch.
"""
from __future__ import annotations

import math

import torch


def _axis_sigma(n: int, lo: int, hi: int, pitch: float, kvac: float, n_bg: float, device) -> torch.Tensor:
    s = torch.zeros(n, dtype=torch.float64)
    for i in range(n):
        if i < lo:
            s[i] = 3.0 * n_bg * math.log(1e4) / (kvac * lo * pitch) * ((lo - i) / lo) ** 2
        elif i >= n - hi:
            s[i] = 3.0 * n_bg * math.log(1e4) / (kvac * hi * pitch) * ((i - (n - hi - 1)) / hi) ** 2
    return s.to(device)


def _wavenumbers(n: int, pitch: float, device):
    p = 2.0 * math.pi * torch.fft.fftfreq(n, d=pitch, dtype=torch.float64)
    q = p.clone()
    if n % 2 == 0:
        q[n // 2] = 0.0
    return p.to(device), q.to(device)


class TorchCBS:
    """Iteration state on one grid: eps_r float (nz, ny, nx) on a CUDA device, the splitting
    (k0^2, epsilon) in SI units, pads per face, x-polarised plane-wave sheet on z = pad_lo[z]
    with amplitude -2 i k_b / pitch."""

    def __init__(self, eps_r: torch.Tensor, pitch: float, lam: float, n_bg: float, pad_lo, pad_hi,
                 k0sq: float, epsilon: float):
        dev = eps_r.device
        nz, ny, nx = eps_r.shape
        kvac = 2.0 * math.pi / lam
        sx = _axis_sigma(nx, pad_lo[0], pad_hi[0], pitch, kvac, n_bg, dev)
        sy = _axis_sigma(ny, pad_lo[1], pad_hi[1], pitch, kvac, n_bg, dev)
        sz = _axis_sigma(nz, pad_lo[2], pad_hi[2], pitch, kvac, n_bg, dev)
        sigma = sz[:, None, None] + sy[None, :, None] + sx[None, None, :]
        k2 = kvac ** 2 * torch.complex(eps_r.double(), sigma)
        kt2 = complex(k0sq, epsilon)
        V = k2 - kt2
        self.V = V.to(torch.complex64)
        self.gamma = ((1j / epsilon) * V).to(torch.complex64)
        px, qx = _wavenumbers(nx, pitch, dev)
        py, qy = _wavenumbers(ny, pitch, dev)
        pz, qz = _wavenumbers(nz, pitch, dev)
        p2 = pz[:, None, None] ** 2 + py[None, :, None] ** 2 + px[None, None, :] ** 2
        q2 = qz[:, None, None] ** 2 + qy[None, :, None] ** 2 + qx[None, None, :] ** 2
        self.inv_a = (1.0 / (p2 - q2 - kt2)).to(torch.complex64)
        self.inv_b = (1.0 / (p2 - kt2)).to(torch.complex64)
        self.q = (qx[None, None, :].float(), qy[None, :, None].float(), qz[:, None, None].float())
        self.S = torch.zeros((3, nz, ny, nx), dtype=torch.complex64, device=dev)
        self.S[0, pad_lo[2]] = complex(0.0, -2.0 * kvac * n_bg / pitch)

    def iterate(self, E: torch.Tensor, n: int) -> torch.Tensor:
        """n iterations from E (updated in place); returns the last ||delta||^2 (float64)."""
        qx, qy, qz = self.q
        r = None
        for _ in range(n):
            W = torch.fft.fftn(self.V * E + self.S, dim=(-3, -2, -1))
            c = (qx * W[0] + qy * W[1] + qz * W[2]) * self.inv_a
            W[0] = (W[0] + qx * c) * self.inv_b
            W[1] = (W[1] + qy * c) * self.inv_b
            W[2] = (W[2] + qz * c) * self.inv_b
            W = torch.fft.ifftn(W, dim=(-3, -2, -1))
            delta = self.gamma * (E - W)
            E -= delta
            r = torch.sum(delta.real.double() ** 2 + delta.imag.double() ** 2)
        return r
