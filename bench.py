#!/usr/bin/env python
"""Benchmark of the GB300 CBS solver: CBS voxel-iterations per second at paper scale.

One step is one design iteration of the paper's method on the design volume of Fig. 4:
621 x 621 x 261 voxels at 177 nm (lambda = 1064 nm) plus absorbing layers
[lambda, lambda, 6 lambda] = [6, 6, 36] voxels per face, padded to the FFT lengths
640 x 640 x 336 (137.6 M voxels), holding the D = 109 um, NA 0.84, n = 1.54 Fresnel lens the
design starts from: set the permittivity (potential and splitting), a forward solve of the
x-polarised plane wave and an adjoint solve of the focal intensity |E(r0)|^2 of --iters
iterations each, and the gradient.  A converged solve on this volume takes of the order of
1e4 iterations; a fixed count keeps a step at the cost of a design iteration's solves and
makes the work per step exact.  The metric is voxels x (forward + adjoint iterations) / time.

After the timed region:
  * "parity": the GPU's forward field, adjoint field and gradient after 2 iterations from zero
    against the FP64 CPU oracle on the full grid (the same legs time "cpu_baseline");
  * "fresnel_lens_275x275x315": one converged design iteration (relative residual --tol) of
    the Fig. 1 lens workload (D = 16 um, NA 0.84, n = 1.5, 275 x 275 x 315 at lambda/16), and
    the same with gentler absorbing layers ("..._gentle_layers": round trip 1e-2, the largest
    overlapping profile in edges and corners), which lower the shift epsilon and the iterations;
  * "cufft_comparison": the same iteration written with cuFFT and element-wise torch kernels;
  * "serving": a seeded request stream over the five serving grid sizes (64^3 .. 384x384x256,
    spheres and lenses, forward and forward + adjoint, gentler layers by default) through the
    continuous-batching server, with the same requests' single-solve times beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

N > 1 runs one independent replica per GPU (launched by torch.distributed.run); the value is
the sum over replicas of voxel-iterations divided by the slowest rank's time.  The
reference arm (--impl reference) times the FP64 CPU oracle on the host cores, one oracle
iteration of the same grid per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2506_15411_gb300 import inputs  # noqa: E402

LAM = 1.064e-6
# headline workload: the paper-scale design volume (Fig. 4)
GRID = (640, 640, 336)
PITCH = 177e-9
PADS = (6, 6, 36)
D_LENS, NA, N_LENS = 109e-6, 0.84, 1.54
ITERS = 200
WORKLOAD = "paper_scale_lens_640x640x336_177nm_fwd200_adj200_grad"
# secondary workload: the Fig. 1 lens, solved to a relative residual
C2_GRID = (275, 275, 315)
C2_PITCH = LAM / 16
C2_LENS = (16e-6, 0.84, 1.5)
C2_WORKLOAD = "fresnel_lens_275x275x315_lambda16_fwd_adj_grad"

METRIC = "CBS voxel-iters/s"
UNIT = "voxel-iter/s"
ORACLE_ITERS = 2     # oracle iterations per solve: CPU baseline and equal-iteration parity
# algorithmic HBM bytes per voxel of each pass (complex64 fields, 3 components, V complex64)
# (k_xpass_fwd runs once per solve; every iteration runs the other four: 248 B per voxel)
PASS_BYTES = {"k_xpass_fwd": 56, "k_ypass_fwd": 48, "k_zpass_green": 48, "k_ypass_inv": 48,
              "k_xpass_inv_fwd": 104}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_paper_scale_640x640x336.json")
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def workload():
    return inputs.fresnel_lens_workload(*GRID, PITCH, LAM, D_LENS, NA, N_LENS, pad_lo=PADS, pad_hi=PADS)


def c2_workload():
    return inputs.fresnel_lens_workload(*C2_GRID, C2_PITCH, LAM, *C2_LENS)


def base_config(wl, iters):
    nx, ny, nz = GRID
    return {"workload": WORKLOAD, "grid_xyz": list(GRID), "voxels": nx * ny * nz,
            "design_volume_xyz": [621, 621, 261],
            "pitch_nm": round(PITCH * 1e9, 3), "lambda_nm": LAM * 1e9, "pads_per_face_xyz": list(PADS),
            "lens": {"D_um": D_LENS * 1e6, "NA": NA, "n": N_LENS}, "focus_voxel_xyz": list(wl.r0),
            "iters_per_solve": iters,
            "l2": "inputs larger than L2 (E, E_adj, W: 3.3 GB each; V 1.1 GB)"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def host_memory_gb():
    """Memory this process may still use on the host (MemAvailable, capped by a cgroup limit)."""
    avail = None
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                avail = int(ln.split()[1]) * 1024
    except Exception:
        pass
    for path in ("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory/memory.limit_in_bytes"):
        try:
            v = open(path).read().strip()
            if v.isdigit():
                lim = int(v)
                used = 0
                for up in ("/sys/fs/cgroup/memory.current", "/sys/fs/cgroup/memory/memory.usage_in_bytes"):
                    try:
                        used = int(open(up).read().strip())
                        break
                    except Exception:
                        pass
                avail = lim - used if avail is None else min(avail, lim - used)
        except Exception:
            pass
    return None if avail is None else avail / 1e9


# peak host memory of the oracle legs on the full grid (FP64 fields of 6.6 GB, FFT work
# arrays and the GPU fields brought back for the comparison), in GB
ORACLE_HOST_GB = 110.0


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={SMI_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for ln in open(self.path):
                f = [x.strip() for x in ln.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
        except Exception:
            pass
        finally:
            try:
                os.remove(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(float(r[1]) for r in rows), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def parity_voxel(wl):
    """Objective voxel of the equal-iteration oracle comparison: on the axis, one voxel past
    the plane-wave sheet.  Two iterations build the field up only within a few voxels of the
    sheet (after two iterations the field falls by about 3x per voxel away from it with this
    grid's shift epsilon = 9.6 k_vac^2), so the focus itself still holds rounding noise."""
    return (GRID[0] // 2, GRID[1] // 2, wl.z_source + 1)


def oracle_design_iteration(wl, iters, r0):
    """FP64 oracle on the full grid: `iters` forward iterations from zero, `iters` adjoint
    iterations of |E(r0)|^2 from zero, the gradient.  Returns a dict with the fields, the
    solve time (set-up excluded) and the worker threads."""
    from oracle import cbs_oracle as co
    g = co.Grid(*GRID, PITCH, LAM, 1.0, wl.pad_lo, wl.pad_hi)
    k2 = co.k_squared(g, wl.eps)
    S = co.plane_wave_source(g)
    sp = co.splitting(k2)
    t = time.perf_counter()
    fwd = co.cbs_solve(g, k2, S, tol=0.0, max_iter=iters, split=sp)
    del S
    Sa = co.adjoint_source(g, fwd.E, r0)
    adj = co.cbs_solve(g, k2, Sa, tol=0.0, max_iter=iters, split=sp)
    dt = time.perf_counter() - t
    del Sa, k2
    grad = co.gradient(g, fwd.E, adj.E)
    return {"E": fwd.E, "Ea": adj.E, "grad": grad, "objective": co.objective(fwd.E, r0),
            "seconds": dt, "iters": 2 * iters, "workers": co.WORKERS, "split": sp}


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle as it stands, one iteration of the full grid per
    step (set-up once, before the warm-up)."""
    if rank != 0:
        return
    from oracle import cbs_oracle as co
    wl = workload()
    N = int(np.prod(GRID))
    g = co.Grid(*GRID, PITCH, LAM, 1.0, wl.pad_lo, wl.pad_hi)
    k2 = co.k_squared(g, wl.eps)
    S = co.plane_wave_source(g)
    sp = co.splitting(k2)
    E = None
    times = []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        r = co.cbs_solve(g, k2, S, tol=0.0, max_iter=1, E0=E, split=sp)
        dt = time.perf_counter() - t
        E = r.E
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = N * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": dict(base_config(wl, args.iters), parallelism="host cores"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": co.WORKERS, "kind": "oracle",
                             "sample": f"one FP64 oracle iteration of the full {GRID[0]}x{GRID[1]}x{GRID[2]} "
                                       "grid per step (scipy.fft workers = cores, NumPy elementwise on one core)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cufft_comparison(plan, eps, wl, iters, stream):
    """The same iteration written with cuFFT and element-wise torch kernels
    (paper_2506_15411_gb300.cufft_reference), timed with CUDA events for `iters` iterations
    after 3, and both paths run 8 iterations from zero to cross-check the iterate."""
    import torch
    from paper_2506_15411_gb300 import PlaneWave
    from paper_2506_15411_gb300.cufft_reference import TorchCBS
    k0sq, epsilon = plan.splitting()
    ref = TorchCBS(eps, PITCH, LAM, 1.0, wl.pad_lo, wl.pad_hi, k0sq, epsilon)
    nz, ny, nx = eps.shape
    Et = torch.zeros((3, nz, ny, nx), dtype=torch.complex64, device=eps.device)
    ref.iterate(Et, 3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ref.iterate(Et, iters)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_iter = e0.elapsed_time(e1) / iters
    K = 8
    Et.zero_()
    ref.iterate(Et, K)
    plan.set_solver(0.0, K, K)
    Eo, _ = plan.forward(PlaneWave())
    torch.cuda.synchronize()
    diff = float(torch.linalg.vector_norm(Eo - Et) / torch.linalg.vector_norm(Et))
    del ref, Et, Eo
    torch.cuda.empty_cache()
    return {"what": "same iteration with torch.fft (cuFFT) 3D FFTs and element-wise torch kernels",
            "ms_per_iteration": ms_iter, "iterations_timed": iters,
            f"rel_diff_after_{K}_iterations": diff}


def combine_ranks(times_ms, counts, world, device):
    """Replicas: the slowest rank's time of each timed region (max) and the work of all ranks
    (sum); with one rank, the inputs.  Returns (times, counts) as lists."""
    import torch
    tmax = torch.tensor(times_ms, dtype=torch.float64, device=device)
    tsum = torch.tensor(counts, dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return tmax.tolist(), tsum.tolist()


def pass_table(passes, N):
    passes = {k: v for k, v in passes.items() if v[1] > 0}   # the per-iteration kernels
    tot = sum(v[0] for v in passes.values())
    return {k: {"avg_ms": v[0] / v[1], "timed_launches": v[1], "share": v[0] / tot,
                "bytes_per_voxel": PASS_BYTES[k],
                "GBps_algorithmic": PASS_BYTES[k] * N / (v[0] / v[1] / 1e3) / 1e9}
            for k, v in passes.items()}


GENTLE_LAYERS = {"layer_round_trip": 1e-2, "layer_corner_max": True}


def secondary_c2(args, stream, dev, layers=None):
    """One converged design iteration of the Fig. 1 lens (set eps, forward and adjoint to
    relative residual args.tol, gradient), after one untimed one; `layers` selects absorbing-
    layer options of the plan (None: the defaults)."""
    import torch
    from paper_2506_15411_gb300 import CBSPlan, PlaneWave
    wl = c2_workload()
    nx, ny, nz = C2_GRID
    N = nx * ny * nz
    eps = torch.from_numpy(wl.eps).to(dev)
    E = torch.empty((3, nz, ny, nx), dtype=torch.complex64, device=dev)
    Ea = torch.empty_like(E)
    grad = torch.empty((nz, ny, nx), dtype=torch.float32, device=dev)
    with CBSPlan(nx, ny, nz, C2_PITCH, LAM, 1.0, wl.pad_lo, wl.pad_hi, tol=args.tol, max_iter=args.max_iter,
                 check_every=64, device=dev, stream=stream, **(layers or {})) as plan:
        def step():
            plan.set_permittivity(eps)
            _, sf = plan.forward(PlaneWave(), E=E)
            _, sa = plan.adjoint(wl.r0, E, Ea)
            _, obj = plan.gradient(E, Ea, wl.r0, grad)
            return sf, sa, obj
        step()
        plan.set_profiling(True)
        plan.pass_times(reset=True)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sf, sa, obj = step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        table = pass_table(plan.pass_times(reset=True), N)
        plan_eps = plan.splitting()[1]
    it = sf.iters + sa.iters
    return {"workload": C2_WORKLOAD, "grid_xyz": list(C2_GRID), "pads_per_face_xyz": list(wl.pad_lo),
            "layers": layers or {"layer_round_trip": 1e-4, "layer_power": 2, "layer_corner_max": False},
            "splitting_epsilon_over_kvac2": plan_eps / (2 * np.pi / LAM) ** 2,
            "tol": args.tol, "ms_fwd_adj_grad": ms, "iters_forward": sf.iters, "iters_adjoint": sa.iters,
            "rel_resid_forward": sf.rel_resid, "rel_resid_adjoint": sa.rel_resid, "objective": obj,
            "voxel_iters_per_s": N * it / (ms / 1e3),
            "iteration_ms": sum(p["avg_ms"] for p in table.values()), "passes": table}


def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2506_15411_gb300 import CBSPlan, PlaneWave

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = workload()
    nx, ny, nz = GRID
    N = nx * ny * nz
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    eps = torch.from_numpy(wl.eps).to(dev)
    E = torch.empty((3, nz, ny, nx), dtype=torch.complex64, device=dev)
    Ea = torch.empty_like(E)
    grad = torch.empty((nz, ny, nx), dtype=torch.float32, device=dev)
    check = max(1, args.iters // 2)
    plan = CBSPlan(nx, ny, nz, PITCH, LAM, 1.0, wl.pad_lo, wl.pad_hi, tol=0.0,
                   max_iter=args.iters, check_every=check, device=dev, stream=stream)
    src = PlaneWave()

    def step():
        plan.set_permittivity(eps)
        _, sf = plan.forward(src, E=E)
        _, sa = plan.adjoint(wl.r0, E, Ea)
        _, obj = plan.gradient(E, Ea, wl.r0, grad)
        return sf, sa, obj

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    # --- device-resident timed region -------------------------------------------------------
    plan.set_profiling(True)
    plan.pass_times(reset=True)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = 0
    launches = 0
    stats = []
    with ClockSampler(local_rank) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            sf, sa, obj = step()
            iters += sf.iters + sa.iters
            # set-up 3 + forward (1 + 4/iter) + adjoint source 1 + adjoint (1 + 4/iter) + gradient 2
            launches += 3 + 1 + 4 * sf.iters + 1 + 1 + 4 * sa.iters + 2
            stats.append((sf, sa, obj))
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    clocks = clk.summary()
    passes = plan.pass_times(reset=True)
    plan.set_profiling(False)
    # --- end to end through the host-buffer API --------------------------------------------
    eps_host = torch.from_numpy(wl.eps).pin_memory()
    grad_host = torch.empty((nz, ny, nx), dtype=torch.float32).pin_memory()
    plan.design_step_host(eps_host.numpy(), src, wl.r0, grad_host.numpy())   # allocate plan buffers
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_iters = 0
    e0.record(stream)
    for _ in range(args.steps):
        _, _, f, a = plan.design_step_host(eps_host.numpy(), src, wl.r0, grad_host.numpy())
        e_iters += f.iters + a.iters
    e1.record(stream)
    barrier()
    e_ms = e0.elapsed_time(e1)

    (ms_max, e_ms_max), (iters_all, e_iters_all) = combine_ranks([ms, e_ms], [float(iters), float(e_iters)],
                                                                 world, dev)
    if rank != 0:
        plan.close()
        return
    value = N * iters_all / (ms_max / 1e3)
    e2e_value = N * e_iters_all / (e_ms_max / 1e3)

    # roofline of the dominant pass (largest share of timed pass time)
    peak, peak_kind = peaks()
    table = pass_table(passes, N)
    dom = max(table, key=lambda k: table[k]["share"])
    avg_ms = table[dom]["avg_ms"]
    achieved = PASS_BYTES[dom] * N / (avg_ms / 1e3) / 1e9
    iter_ms = sum(p["avg_ms"] for p in table.values())
    sf, sa, obj = stats[-1]
    cfg = base_config(wl, args.iters)
    cfg.update({"iters_forward": sf.iters, "iters_adjoint": sa.iters, "rel_resid_forward": sf.rel_resid,
                "rel_resid_adjoint": sa.rel_resid, "objective": obj, "parallelism": f"replicas x{world}",
                "iteration_ms": iter_ms, "iteration_GBps_248B": 248 * N / (iter_ms / 1e3) / 1e9,
                "iteration_frac_248B": 248 * N / (iter_ms / 1e3) / 1e9 / peak,
                "iteration_frac_280B_model": 280 * N / (iter_ms / 1e3) / 1e9 / peak,
                "passes": table, "check_every": check})

    # --- after the timed region: oracle parity and CPU baseline ------------------------------
    cpu = None
    parity = None
    if not args.no_cpu_baseline:
        mem = host_memory_gb()
        if mem is not None and mem < ORACLE_HOST_GB:
            parity = {"skipped": f"host memory available {mem:.0f} GB < {ORACLE_HOST_GB:.0f} GB the FP64 "
                                 "oracle of the full grid needs"}
        else:
            rp = parity_voxel(wl)
            plan.set_permittivity(eps)
            plan.set_solver(0.0, ORACLE_ITERS, ORACLE_ITERS)
            Eg, _ = plan.forward(src)
            Eag, _ = plan.adjoint(rp, Eg)
            gg, objg = plan.gradient(Eg, Eag, rp)
            torch.cuda.synchronize(dev)
            Eg_h, Eag_h, gg_h = Eg.cpu().numpy(), Eag.cpu().numpy(), gg.cpu().numpy()
            del Eg, Eag, gg
            o = oracle_design_iteration(wl, ORACLE_ITERS, rp)
            rate = N * o["iters"] / o["seconds"]
            cpu = {"value": rate, "unit": UNIT, "cores": o["workers"], "kind": "oracle",
                   "sample": f"{ORACLE_ITERS} forward + {ORACLE_ITERS} adjoint FP64 oracle iterations from zero "
                             f"of the full {nx}x{ny}x{nz} grid ({o['seconds']:.1f} s; scipy.fft workers = cores, "
                             "NumPy elementwise on one core)"}
            k0g, epg = plan.splitting()
            parity = {"against": "FP64 oracle, equal iteration count from zero, full grid",
                      "iterations_per_solve": ORACLE_ITERS, "objective_voxel_xyz": list(rp),
                      "field_rel_l2": rel_l2(Eg_h, o["E"]),
                      "adjoint_field_rel_l2": rel_l2(Eag_h, o["Ea"]),
                      "gradient_rel_l2": rel_l2(gg_h, o["grad"]),
                      "objective_rel": abs(objg - o["objective"]) / abs(o["objective"]),
                      "splitting_rel": [abs(k0g - o["split"].k0sq) / abs(o["split"].k0sq),
                                        abs(epg - o["split"].epsilon) / o["split"].epsilon]}
            del o, Eg_h, Eag_h, gg_h
    cufft = None
    if args.cufft_iters > 0:
        cufft = cufft_comparison(plan, eps, wl, args.cufft_iters, stream)
        cufft["ours_ms_per_iteration"] = iter_ms
        cufft["speedup_of_fused_kernels"] = cufft["ms_per_iteration"] / iter_ms
    plan.close()
    del E, Ea, grad, eps
    torch.cuda.empty_cache()
    c2 = secondary_c2(args, stream, dev) if args.c2 and args.tol > 0 else None
    c2g = secondary_c2(args, stream, dev, GENTLE_LAYERS) if args.c2 and args.tol > 0 else None
    serving = None
    if args.serve_requests > 0 and args.tol > 0:
        # served-solve latency (the metric's third part): a seeded stream over the five grid
        # sizes of the serving workload through the continuous-batching server, each request
        # also solved alone for the single-solve percentiles
        from paper_2506_15411_gb300.serve import measure_stream
        serving = measure_stream(args.serve_requests, [inputs.parse_size(v) for v in args.serve_sizes],
                                 tol=args.tol, layers=args.serve_layers)
    traffic = load_traffic(dom)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic", "config": cfg,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
                         "traffic": traffic,
                         "algorithmic_bytes_per_launch": PASS_BYTES[dom] * N},
            "cpu_baseline": cpu, "parity": parity,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * N,
                    "d2h_bytes_per_step": 4 * N + 8, "ms_per_step": e_ms_max / args.steps},
            "gpu_launches": launches * world, "clocks": clocks,
            "fresnel_lens_275x275x315": c2, "fresnel_lens_275x275x315_gentle_layers": c2g,
            "serving": serving, "cufft_comparison": cufft}
    print(json.dumps(line), flush=True)


def source_digest():
    """sha256 over the CUDA sources (kernels, headers), to tell whether measured counters are
    still those of the code being run."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2506_15411_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def load_traffic(kernel, path=TRAFFIC_FILE):
    """DRAM bytes per launch of `kernel` on the headline workload from the committed ncu
    summary, or None when the kernels have changed since those counters were taken."""
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("source_sha256") != source_digest():
            return None
        v = d["bytes_per_launch"].get(kernel)
        return None if v is None else float(v)
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--iters", type=int, default=ITERS, help="iterations of each solve of a step")
    ap.add_argument("--tol", type=float, default=1e-4, help="relative residual of the converged lens leg")
    ap.add_argument("--max-iter", type=int, default=200000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-c2", dest="c2", action="store_false",
                    help="skip the converged 275x275x315 lens design iteration")
    ap.add_argument("--serve-requests", type=int, default=20,
                    help="requests of the served-latency stream after the timed region (0: none; "
                         "skipped when --tol <= 0)")
    ap.add_argument("--serve-sizes", nargs="+", default=["64", "128", "192x192x128", "256x256x192", "384x384x256"],
                    help="grid sizes of that stream")
    ap.add_argument("--serve-layers", choices=["default", "gentle"], default="gentle",
                    help="absorbing layers of the stream's requests")
    ap.add_argument("--cufft-iters", type=int, default=20,
                    help="iterations of the cuFFT comparison timed after the timed region (0: none)")
    ap.add_argument("--print-digest", action="store_true", help="print the CUDA source digest and exit")
    args = ap.parse_args()
    if args.print_digest:
        print(source_digest())
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
