"""Solve time against grid size: the resolution sweep of Fig. 1(b) on the CUDA solver.

The D = 16 um Fresnel lens (NA 0.84, n = 1.5, lambda = 1064 nm) in the physical domain of the
275 x 275 x 315 workload (interior 16.16 x 16.16 x 8.18 um, absorbing layers [lambda, lambda,
6 lambda] per face) is solved at pitches lambda/6 ... lambda/18; each axis is rounded up to the
next length the FFTs support (prime factors 2, 3, 5, 7, 11, 13), the extra voxels joining the
background interior.  One JSON line per pitch: grid, voxels, forward iterations to the
relative residual --tol, seconds (host wall time of the solve, permittivity set-up excluded),
time per iteration and voxel-iterations per second; a last line fits t = c N^a over the
sweep.  --layers gentle uses the gentler absorbing layers (round trip 1e-2, the largest
profile where layers overlap) instead of the defaults.

    python -m paper_2506_15411_gb300.sweep --ppl 6 8 10 12 14 16 18 [--layers gentle]
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch

from . import inputs
from .solver import CBSPlan, PlaneWave

LAM = 1.064e-6
INTERIOR_XY_UM = 243 * LAM / 16 * 1e6      # the 275^2 x 315 lens grid without its layers
INTERIOR_Z_UM = 123 * LAM / 16 * 1e6
D_UM, NA, N_LENS = 16.0, 0.84, 1.5


def fft_size(n: int) -> int:
    """Smallest m >= n whose prime factors are all in {2, 3, 5, 7, 11, 13}."""
    m = n
    while True:
        r = m
        for p in (2, 3, 5, 7, 11, 13):
            while r % p == 0:
                r //= p
        if r == 1:
            return m
        m += 1


def grid_for(ppl: int):
    pitch = LAM / ppl
    pads = (ppl, ppl, 6 * ppl)
    nxy = fft_size(int(math.ceil(INTERIOR_XY_UM * 1e-6 / pitch)) + 2 * pads[0])
    nz = fft_size(int(math.ceil(INTERIOR_Z_UM * 1e-6 / pitch)) + 2 * pads[2])
    return nxy, nxy, nz, pitch, pads


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ppl", type=int, nargs="+", default=[6, 8, 10, 12, 14, 16, 18])
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--check-every", type=int, default=64)
    ap.add_argument("--layers", choices=["default", "gentle"], default="default")
    args = ap.parse_args()
    layers = {"layer_round_trip": 1e-2, "layer_corner_max": True} if args.layers == "gentle" else {}
    rows = []
    for ppl in args.ppl:
        nx, ny, nz, pitch, pads = grid_for(ppl)
        wl = inputs.fresnel_lens_workload(nx, ny, nz, pitch, LAM, D_UM * 1e-6, NA, N_LENS, pad_lo=pads, pad_hi=pads)
        with CBSPlan(nx, ny, nz, pitch, LAM, 1.0, pads, pads, tol=args.tol, max_iter=200000,
                     check_every=args.check_every, **layers) as plan:
            plan.set_permittivity(torch.from_numpy(wl.eps).to(plan.device))
            E, st = plan.forward(PlaneWave())          # warm-up of graphs and clocks
            E, st = plan.forward(PlaneWave(), E=E)
            torch.cuda.synchronize()
        N = nx * ny * nz
        row = {"ppl": ppl, "layers": args.layers, "pitch_nm": pitch * 1e9, "grid": [nx, ny, nz], "voxels": N,
               "iters": st.iters,
               "status": st.status, "seconds": st.seconds, "ms_per_iter": 1e3 * st.seconds / st.iters,
               "voxel_iters_per_s": N * st.iters / st.seconds}
        rows.append(row)
        print(json.dumps(row), flush=True)
    if len(rows) >= 2:
        lx = np.log([r["voxels"] for r in rows])
        a_t, _ = np.polyfit(lx, np.log([r["seconds"] for r in rows]), 1)
        a_i, _ = np.polyfit(lx, np.log([r["ms_per_iter"] for r in rows]), 1)
        print(json.dumps({"fit": "t = c N^a", "a_solve": a_t, "a_per_iteration": a_i,
                          "N_range": [rows[0]["voxels"], rows[-1]["voxels"]]}), flush=True)


if __name__ == "__main__":
    main()
