"""The cuFFT comparison iteration (paper_2506_15411_gb300/cufft_reference.py, torch.fft +
element-wise torch) against the FP64 oracle at equal iteration count, on the CPU.  It is a
measurement baseline beside the fused kernels, so it must compute the same series."""
from __future__ import annotations

import numpy as np
import torch

from oracle import cbs_oracle as co
from paper_2506_15411_gb300 import inputs
from paper_2506_15411_gb300.cufft_reference import TorchCBS

LAM = 1.064e-6


def test_torch_iteration_matches_the_oracle():
    g = co.Grid(20, 18, 24, LAM / 8, LAM, 1.0, (3, 2, 4), (2, 3, 4))
    eps = inputs.random_eps(g.nx, g.ny, g.nz, seed=17)
    K = 12
    ref = co.forward(g, eps, co.plane_wave_source(g), tol=0.0, max_iter=K)
    sp = ref.split
    t = TorchCBS(torch.from_numpy(eps), g.pitch, LAM, 1.0, g.pad_lo, g.pad_hi, sp.k0sq, sp.epsilon)
    E = torch.zeros((3,) + g.shape, dtype=torch.complex64)
    r = t.iterate(E, K)
    err = np.linalg.norm(E.numpy() - ref.E) / np.linalg.norm(ref.E)
    assert err <= 2e-5, err
    assert abs(float(r) ** 0.5 - ref.history[-1]) <= 1e-4 * ref.history[-1]
