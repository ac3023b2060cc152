"""Inverse design of the lens thickness map (Section 3, Fig. 2(a)) on the CUDA solver.

    h_eff = G_sigma[M h] -> eps_r (subpixel shape Theta(h - z)) -> forward / adjoint CBS
    -> dL/d eps_r -> dL/dh (chain rule) -> Adam ascent on L = |E(r0)|^2

h is a float32 (ny, nx) map in micrometres on the plan's device.  Every step runs in
libcbs.so (cbs_design_* in include/cbs.h); this module marshals arguments and keeps the
fields between steps so that each solve can start from the previous step's solution.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import List, Optional

import torch

from . import _lib as L
from .solver import CBSPlan, Stats, _field_like, _ptr, _stats


@dataclass
class StepInfo:
    objective: float
    fwd: Stats
    adj: Stats
    seconds: float


class Design:
    """The design pipeline of one plan: mirror symmetry, optional Gaussian smoothing
    (sigma_um), subpixel shape above z_base, Adam (alpha in micrometres) with
    0 <= h <= h_max_um inside the aperture of diameter aperture_um and h = 0 outside."""

    def __init__(self, plan: CBSPlan, z_base: int, n_lens: float, aperture_um: float, h_max_um: float,
                 sigma_um: float = 0.0, mirror: bool = True, alpha: float = 0.3, beta1: float = 0.9,
                 beta2: float = 0.999, adam_eps: float = 1e-6):
        self.plan = plan
        self.lib = plan.lib
        self.params = dict(z_base=int(z_base), n_lens=float(n_lens), aperture_um=float(aperture_um),
                           h_max_um=float(h_max_um), sigma_um=float(sigma_um), mirror=bool(mirror),
                           alpha=float(alpha), beta1=float(beta1), beta2=float(beta2), adam_eps=float(adam_eps))
        d = L.cbs_design_desc(int(z_base), float(n_lens), float(aperture_um), float(h_max_um), float(sigma_um),
                              1 if mirror else 0, float(alpha), float(beta1), float(beta2), float(adam_eps))
        h = ctypes.c_void_p()
        L.check(self.lib.cbs_design_create(ctypes.byref(h), plan.handle, ctypes.byref(d)))
        self.handle = h
        self.map_shape = (plan.ny, plan.nx)
        self.E: Optional[torch.Tensor] = None
        self.E_adj: Optional[torch.Tensor] = None

    def close(self):
        if getattr(self, "handle", None):
            self.lib.cbs_design_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check_map(self, h: torch.Tensor, name: str):
        if h.dtype != torch.float32 or tuple(h.shape) != self.map_shape or not h.is_contiguous() \
                or h.device != self.plan.device:
            raise ValueError(f"{name} must be a contiguous float32 {self.map_shape} tensor on {self.plan.device}")

    def reset(self):
        L.check(self.lib.cbs_design_reset(self.handle))

    def state_dict(self, h: torch.Tensor, fields: bool = False) -> dict:
        """The loop's state for a checkpoint: the map h, Adam's moments m and v, the step
        count t, the design parameters and the plan's grid; with fields=True also the last
        forward and adjoint fields, so that a warm-started next step resumes exactly."""
        self._check_map(h, "h")
        m = torch.empty(self.map_shape, dtype=torch.float32, device=self.plan.device)
        v = torch.empty_like(m)
        t = ctypes.c_int()
        L.check(self.lib.cbs_design_get_state(self.handle, ctypes.c_void_p(_ptr(m)), ctypes.c_void_p(_ptr(v)),
                                              ctypes.byref(t)))
        state = {"h": h.detach().clone(), "m": m, "v": v, "t": t.value, "params": dict(self.params),
                 "grid": tuple(self.plan.shape)}
        if fields and self.E is not None:
            state["E"] = self.E.clone()
            state["E_adj"] = self.E_adj.clone()
        return state

    def load_state_dict(self, state: dict) -> torch.Tensor:
        """Restore a state_dict() into this object (same grid and parameters) and return the
        map h on the plan's device; the next step continues as the saved loop would have."""
        if tuple(state["grid"]) != tuple(self.plan.shape) or state["params"] != self.params:
            raise ValueError("checkpoint is of another grid or design parameters")
        dev = self.plan.device
        h = state["h"].to(device=dev, dtype=torch.float32).contiguous()
        m = state["m"].to(device=dev, dtype=torch.float32).contiguous()
        v = state["v"].to(device=dev, dtype=torch.float32).contiguous()
        for name, x in (("h", h), ("m", m), ("v", v)):
            self._check_map(x, name)
        L.check(self.lib.cbs_design_set_state(self.handle, ctypes.c_void_p(_ptr(m)), ctypes.c_void_p(_ptr(v)),
                                              int(state["t"])))
        if "E" in state:
            self.E = state["E"].to(dev).contiguous()
            self.E_adj = state["E_adj"].to(dev).contiguous()
        else:
            self.E = self.E_adj = None
        return h

    def save(self, path: str, h: torch.Tensor, fields: bool = False):
        """Write state_dict(h, fields) to path (torch.save, tensors moved to the host)."""
        st = self.state_dict(h, fields)
        torch.save({k: (x.cpu() if isinstance(x, torch.Tensor) else x) for k, x in st.items()}, path)

    def load(self, path: str) -> torch.Tensor:
        """Restore a checkpoint written by save(); returns h on the plan's device."""
        return self.load_state_dict(torch.load(path, map_location="cpu", weights_only=True))

    def permittivity(self, h: torch.Tensor):
        """(eps_r float32 (nz, ny, nx), h_eff float32 (ny, nx)) of the map h."""
        self._check_map(h, "h")
        eps = torch.empty(self.plan.shape, dtype=torch.float32, device=self.plan.device)
        he = torch.empty(self.map_shape, dtype=torch.float32, device=self.plan.device)
        L.check(self.lib.cbs_design_permittivity(self.handle, ctypes.c_void_p(_ptr(h)), ctypes.c_void_p(_ptr(he)),
                                                 ctypes.c_void_p(_ptr(eps))))
        return eps, he

    def height_gradient(self, h: torch.Tensor, grad_eps: torch.Tensor) -> torch.Tensor:
        """dL/dh from dL/d eps_r at the map h."""
        self._check_map(h, "h")
        if grad_eps.dtype != torch.float32 or tuple(grad_eps.shape) != self.plan.shape or not grad_eps.is_contiguous():
            raise ValueError("grad_eps must be a contiguous float32 (nz, ny, nx) tensor")
        gh = torch.empty(self.map_shape, dtype=torch.float32, device=self.plan.device)
        L.check(self.lib.cbs_design_height_gradient(self.handle, ctypes.c_void_p(_ptr(h)),
                                                    ctypes.c_void_p(_ptr(grad_eps)), ctypes.c_void_p(_ptr(gh))))
        return gh

    def adam(self, h: torch.Tensor, grad_h: torch.Tensor):
        """One constrained Adam ascent step on h in place."""
        self._check_map(h, "h")
        self._check_map(grad_h, "grad_h")
        L.check(self.lib.cbs_design_adam(self.handle, ctypes.c_void_p(_ptr(h)), ctypes.c_void_p(_ptr(grad_h))))

    def step(self, h: torch.Tensor, source, r0, warm_start: int = 0, grad_h: Optional[torch.Tensor] = None) -> StepInfo:
        """One design iteration on h (updated in place).  warm_start 1 or 2 starts both
        solves from the previous step's fields (2: residuals relative to a start from zero,
        so they stop early); grad_h, if given, receives dL/dh."""
        self._check_map(h, "h")
        if self.E is None:
            self.E = _field_like(self.plan.shape, self.plan.device)
            self.E_adj = _field_like(self.plan.shape, self.plan.device)
            warm_start = 0
        if grad_h is not None:
            self._check_map(grad_h, "grad_h")
        s = self.plan._source(source, False)
        s.warm_start = int(warm_start)
        r = (ctypes.c_int * 3)(*[int(v) for v in r0])
        obj = ctypes.c_double()
        f, a = L.cbs_stats(), L.cbs_stats()
        L.check(self.lib.cbs_design_step(
            self.handle, ctypes.c_void_p(_ptr(h)), ctypes.byref(s), ctypes.byref(r), ctypes.c_void_p(_ptr(self.E)),
            ctypes.c_void_p(_ptr(self.E_adj)), ctypes.c_void_p(_ptr(grad_h)) if grad_h is not None else None,
            ctypes.byref(obj), ctypes.byref(f), ctypes.byref(a)))
        fs, as_ = _stats(f), _stats(a)
        return StepInfo(obj.value, fs, as_, fs.seconds + as_.seconds)

    def run(self, h: torch.Tensor, source, r0, steps: int, warm_start: int = 2) -> List[StepInfo]:
        """`steps` design iterations; the first starts both solves from zero."""
        out = []
        for k in range(steps):
            out.append(self.step(h, source, r0, warm_start=warm_start if k > 0 else 0))
        return out


class HeightToPermittivity(torch.autograd.Function):
    """eps_r(h) with backward dL/dh = M G_sigma [surface derivative of dL/d eps_r]."""

    @staticmethod
    def forward(ctx, h: torch.Tensor, design: Design):
        hc = h.detach().to(torch.float32).contiguous()
        eps, _ = design.permittivity(hc)
        ctx.design = design
        ctx.save_for_backward(hc)
        return eps

    @staticmethod
    def backward(ctx, grad_eps):
        (hc,) = ctx.saved_tensors
        return ctx.design.height_gradient(hc, grad_eps.to(torch.float32).contiguous()), None


def height_to_permittivity(h: torch.Tensor, design: Design) -> torch.Tensor:
    """Differentiable eps_r (nz, ny, nx) of the thickness map h (ny, nx) [um]; compose with
    autograd.focal_intensity for dL/dh."""
    return HeightToPermittivity.apply(h, design)


def main():
    """Run the design loop on a Fresnel-lens start:

        python -m paper_2506_15411_gb300.design --grid 256 256 192 --ppl 8 --pads 8 8 24 \\
            --D-um 25 --steps 5

    prints one JSON line per step (objective, iterations, seconds).  --checkpoint PATH saves
    h, Adam's state and the fields after every step; --resume PATH continues from one."""
    import argparse
    import json
    import math
    import time

    import numpy as np

    from . import inputs
    from .solver import PlaneWave

    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, nargs=3, required=True, metavar=("NX", "NY", "NZ"))
    ap.add_argument("--lam-nm", type=float, default=1064.0)
    ap.add_argument("--ppl", type=float, default=None, help="voxels per wavelength (else --pitch-nm)")
    ap.add_argument("--pitch-nm", type=float, default=177.0)
    ap.add_argument("--pads", type=int, nargs=3, required=True, help="absorbing voxels per face (x, y, z)")
    ap.add_argument("--D-um", type=float, required=True)
    ap.add_argument("--NA", type=float, default=0.84)
    ap.add_argument("--n-lens", type=float, default=1.54)
    ap.add_argument("--sigma-um", type=float, default=0.355)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--max-iter", type=int, default=200000)
    ap.add_argument("--warm", type=int, default=2)
    ap.add_argument("--checkpoint", default=None, help="write the loop's state here after every step")
    ap.add_argument("--resume", default=None, help="start from a checkpoint written by --checkpoint")
    ap.add_argument("--check-every", type=int, default=64)
    ap.add_argument("--pass-times", action="store_true",
                    help="time the solver's passes with CUDA events and print their averages at the end")
    args = ap.parse_args()
    nx, ny, nz = args.grid
    lam = args.lam_nm * 1e-9
    pitch = lam / args.ppl if args.ppl else args.pitch_nm * 1e-9
    p_um = pitch * 1e6
    z_base = args.pads[2] + 2
    x = inputs.centred_coords(nx, p_um)
    y = inputs.centred_coords(ny, p_um)
    r = np.sqrt(x[None, :] ** 2 + y[:, None] ** 2)
    h_max = args.lam_nm * 1e-3 / (args.n_lens - 1.0)
    h0 = inputs.fresnel_height(r, args.lam_nm * 1e-3, args.D_um, args.NA, args.n_lens).astype(np.float32)
    zf = z_base + int(round(inputs.focal_length(args.D_um, args.NA) / p_um))
    if zf >= nz - args.pads[2]:
        raise SystemExit(f"focus z = {zf} falls in the absorbing layer")
    r0 = (nx // 2, ny // 2, zf)
    with CBSPlan(nx, ny, nz, pitch, lam, 1.0, tuple(args.pads), tuple(args.pads), tol=args.tol,
                 max_iter=args.max_iter, check_every=args.check_every) as plan:
        if args.pass_times:
            plan.set_profiling(True)
        with Design(plan, z_base, args.n_lens, args.D_um, h_max, args.sigma_um) as d:
            h = torch.from_numpy(h0).to(plan.device)
            if args.resume:
                h = d.load(args.resume)
            for k in range(args.steps):
                t0 = time.perf_counter()
                info = d.step(h, PlaneWave(), r0, warm_start=args.warm if k > 0 or args.resume else 0)
                if args.checkpoint:
                    d.save(args.checkpoint, h, fields=True)
                torch.cuda.synchronize()
                print(json.dumps({"step": k, "objective": info.objective, "fwd_iters": info.fwd.iters,
                                  "adj_iters": info.adj.iters, "fwd_status": info.fwd.status,
                                  "adj_status": info.adj.status, "seconds": time.perf_counter() - t0,
                                  "solve_seconds": info.seconds,
                                  "ms_per_iter": 1e3 * info.seconds / max(1, info.fwd.iters + info.adj.iters),
                                  "grid": [nx, ny, nz], "pitch_nm": pitch * 1e9}), flush=True)
                if not math.isfinite(info.objective):
                    raise SystemExit("non-finite objective")
        if args.pass_times:
            t = plan.pass_times()
            print(json.dumps({"pass_avg_ms": {k: v[0] / max(1, v[1]) for k, v in t.items()},
                              "timed_launches": {k: v[1] for k, v in t.items()}}), flush=True)


if __name__ == "__main__":
    main()
