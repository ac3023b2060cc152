"""Run a fixed number of CBS iterations on a synthetic grid, for profilers (ncu) and quick
timing: a seeded random permittivity in [1, 2.25], absorbing layers of one wavelength per
face (pitch lambda/8 by default), an x-polarised plane wave.

    python -m paper_2506_15411_gb300.profile_case --grid 256 256 192 --iters 8

Prints the per-pass event times of the run (CUDA events on the plan's stream).
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import inputs
from .solver import CBSPlan, PlaneWave

LAM = 1.064e-6


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, nargs=3, default=[256, 256, 192], metavar=("NX", "NY", "NZ"))
    ap.add_argument("--iters", type=int, default=8)
    ap.add_argument("--ppl", type=int, default=8, help="voxels per wavelength")
    ap.add_argument("--check-every", type=int, default=8)
    args = ap.parse_args()
    nx, ny, nz = args.grid
    pitch = LAM / args.ppl
    pad = args.ppl
    eps = torch.from_numpy(inputs.random_eps(nx, ny, nz, seed=5)).cuda()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    with CBSPlan(nx, ny, nz, pitch, LAM, 1.0, (pad,) * 3, (pad,) * 3, tol=0.0, max_iter=args.iters,
                 check_every=args.check_every, stream=stream) as plan:
        plan.set_permittivity(eps)
        plan.set_profiling(True)
        E, st = plan.forward(PlaneWave())
        torch.cuda.synchronize()
        t = plan.pass_times()
    n = nx * ny * nz
    print(json.dumps({"grid": [nx, ny, nz], "iters": st.iters, "rel_resid": st.rel_resid,
                      "pass_avg_ms": {k: v[0] / max(1, v[1]) for k, v in t.items()},
                      "voxels": n, "finite": bool(np.isfinite(st.rel_resid))}))


if __name__ == "__main__":
    main()
