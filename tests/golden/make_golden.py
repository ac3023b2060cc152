"""Write the stored expected values of the converged-solve parity tests.

Calls only the FP64 oracle (oracle/) and the seeded input generators; nothing here touches
the CUDA path.  Run from the repository root:

    python tests/golden/make_golden.py            # all fixtures
    python tests/golden/make_golden.py c1_sphere  # one fixture

Fixture c1_sphere: the dielectric-sphere workload (64^3 grid with its absorbing layers of
one wavelength per face, lambda = 1064 nm, pitch lambda/8, sphere n = 1.5 of radius
1.5 um centred in n = 1.0, x-polarised plane wave along +z from the first interior plane),
solved to relative residual 1e-6.  Stored: the iteration count, the final relative residual,
||E||_2 over the grid and E at 1024 voxels drawn with seed 7 (complex, x/y/z components,
9 significant digits).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import cbs_oracle as co  # noqa: E402
from paper_2506_15411_gb300 import inputs  # noqa: E402

LAM = 1.064e-6


def c1_sphere():
    n = 64
    pitch = LAM / 8
    grid = co.Grid(n, n, n, pitch, LAM, 1.0, (8, 8, 8), (8, 8, 8))
    eps = inputs.sphere_eps(n, n, n, pitch, 1.5e-6, 1.5, 1.0)
    S = co.plane_wave_source(grid)
    t = time.time()
    res = co.forward(grid, eps, S, tol=1e-6, max_iter=50000)
    rng = np.random.default_rng(7)
    flat = rng.choice(grid.n_vox, size=4096, replace=False)[:1024]
    z, rem = np.divmod(flat, n * n)
    y, x = np.divmod(rem, n)
    vals = res.E[:, z, y, x]
    return {
        "config": {"nx": n, "ny": n, "nz": n, "pitch_m": pitch, "lambda_m": LAM, "n_bg": 1.0,
                   "pad_lo": [8, 8, 8], "pad_hi": [8, 8, 8], "sphere_radius_m": 1.5e-6,
                   "n_sphere": 1.5, "tol": 1e-6, "source": "plane wave x-pol, z_plane = pad_lo[z]"},
        "iters": res.iters,
        "rel_resid": res.rel_resid,
        "norm_E": float(np.sqrt(np.sum(np.abs(res.E) ** 2))),
        "k0sq": res.split.k0sq,
        "epsilon": res.split.epsilon,
        "voxels_xyz": np.stack([x, y, z], 1).tolist(),
        "E_re": [[float(f"{v:.9g}") for v in row] for row in vals.real.T],
        "E_im": [[float(f"{v:.9g}") for v in row] for row in vals.imag.T],
        "oracle_seconds": time.time() - t,
    }


FIXTURES = {"c1_sphere": c1_sphere}

if __name__ == "__main__":
    names = sys.argv[1:] or list(FIXTURES)
    for name in names:
        data = FIXTURES[name]()
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(data, f)
        print(name, data["iters"], data["rel_resid"], f"{data['oracle_seconds']:.0f}s")
