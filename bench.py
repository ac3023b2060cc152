#!/usr/bin/env python
"""Benchmark of the GB300 CBS solver: CBS voxel-iterations per second.

One step is one design iteration of the paper's method on the Fresnel-lens workload
(D = 16 um, NA 0.84, lambda = 1064 nm, n = 1.5 on n = 1.0, 275 x 275 x 315 voxels at
lambda/16 with absorbing layers [lambda, lambda, 6 lambda] = [16, 16, 96] voxels per face):
set the permittivity (potential and splitting), forward solve of the x-polarised plane wave
to the relative residual --tol, adjoint solve for the focal intensity |E(r0)|^2, gradient.
The metric is voxels x (forward + adjoint iterations) / time; ms_per_step is the forward +
adjoint + gradient time.  After the timed region the same iteration written with cuFFT and
element-wise torch kernels is timed on the same grid ("cufft_comparison"), and a short
seeded request stream (12 requests of 64^3 and 128^3 grids by default) runs through the
continuous-batching server, its p50 / p99 latency and solves/s going into "serving".

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
GRID = (275, 275, 315)
PITCH = LAM / 16
D_LENS, NA, N_LENS = 16e-6, 0.84, 1.5
METRIC = "CBS voxel-iters/s"
ORACLE_ITERS = 2     # oracle iterations of the full grid: CPU baseline and equal-iteration parity
UNIT = "voxel-iter/s"
WORKLOAD = "fresnel_lens_275x275x315_lambda16_fwd_adj_grad"
# algorithmic HBM bytes per voxel of each pass (complex64 fields, 3 components, V complex64)
# (k_xpass_fwd runs once per solve; every iteration runs the other four: 248 B per voxel)
PASS_BYTES = {"k_xpass_fwd": 56, "k_ypass_fwd": 48, "k_zpass_green": 48, "k_ypass_inv": 48,
              "k_xpass_inv_fwd": 104}
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def workload():
    return inputs.fresnel_lens_workload(*GRID, PITCH, LAM, D_LENS, NA, N_LENS)


def base_config(wl, tol):
    nx, ny, nz = GRID
    return {"workload": WORKLOAD, "grid_xyz": list(GRID), "voxels": nx * ny * nz,
            "pitch_nm": round(PITCH * 1e9, 3), "lambda_nm": LAM * 1e9, "pads_per_face_xyz": list(wl.pad_lo),
            "lens": {"D_um": D_LENS * 1e6, "NA": NA, "n": N_LENS}, "focus_voxel_xyz": list(wl.r0),
            "tol": tol, "l2": "inputs larger than L2 (E, E_adj, W: 572 MB each; V 191 MB)"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


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


def cpu_oracle_iteration_rate(wl, iters=1, want_field=False):
    """FP64 oracle, `iters` iterations from zero (after its set-up) on the full grid:
    (voxel-iters/s, seconds, worker threads[, field])."""
    from oracle import cbs_oracle as co
    g = co.Grid(*GRID, PITCH, LAM, 1.0, wl.pad_lo, wl.pad_hi)
    k2 = co.k_squared(g, wl.eps)
    S = co.plane_wave_source(g)
    t = time.perf_counter()
    r = co.cbs_solve(g, k2, S, tol=0.0, max_iter=iters)
    dt = time.perf_counter() - t
    out = (g.n_vox * iters / dt, dt, co.WORKERS)
    return out + (r.E,) if want_field else out


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle as it stands, one iteration per step."""
    if rank != 0:
        return
    wl = workload()
    N = int(np.prod(GRID))
    for _ in range(args.warmup):
        cpu_oracle_iteration_rate(wl)
    times = []
    cores = 1
    for _ in range(args.steps):
        _, dt, cores = cpu_oracle_iteration_rate(wl)
        times.append(dt)
    total = sum(times)
    value = N * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": dict(base_config(wl, args.tol), parallelism="host cores"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "one FP64 oracle iteration of the full 275x275x315 grid per step "
                                       "(scipy.fft workers = cores, NumPy elementwise on one core)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cufft_comparison(plan, eps, wl, iters, stream):
    """The same iteration written with cuFFT and element-wise torch kernels
    (paper_2506_15411_gb300.cufft_reference), timed with CUDA events for `iters` iterations
    after 3, and both paths run 24 iterations from zero to cross-check the iterate."""
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
    K = 24
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
            "rel_diff_after_24_iterations": diff}


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
    plan = CBSPlan(nx, ny, nz, PITCH, LAM, 1.0, wl.pad_lo, wl.pad_hi, tol=args.tol,
                   max_iter=args.max_iter, check_every=args.check_every, device=dev, stream=stream)
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
    cufft = None
    if rank == 0 and args.cufft_iters > 0:
        cufft = cufft_comparison(plan, eps, wl, args.cufft_iters, stream)
    E_k = None
    if rank == 0 and not args.no_cpu_baseline:
        # the GPU iterate after ORACLE_ITERS iterations from zero, for the oracle comparison
        plan.set_solver(0.0, ORACLE_ITERS, ORACLE_ITERS)
        Eg, _ = plan.forward(src)
        E_k = Eg.cpu().numpy()
    if rank != 0:
        plan.close()
        return
    value = N * iters_all / (ms_max / 1e3)
    e2e_value = N * e_iters_all / (e_ms_max / 1e3)

    # roofline of the dominant pass (largest share of timed pass time)
    peak, peak_kind = peaks()
    passes = {k: v for k, v in passes.items() if v[1] > 0}   # the per-iteration kernels
    tot = {k: v[0] for k, v in passes.items()}
    dom = max(tot, key=tot.get)
    avg_ms = passes[dom][0] / passes[dom][1]
    achieved = PASS_BYTES[dom] * N / (avg_ms / 1e3) / 1e9
    traffic = load_traffic(dom)
    pass_table = {k: {"avg_ms": v[0] / v[1], "timed_launches": v[1], "share": tot[k] / sum(tot.values()),
                      "bytes_per_voxel": PASS_BYTES[k],
                      "GBps_algorithmic": PASS_BYTES[k] * N / (v[0] / v[1] / 1e3) / 1e9}
                  for k, v in passes.items()}
    iter_ms = sum(p["avg_ms"] for p in pass_table.values())

    cpu = None
    parity = None
    if not args.no_cpu_baseline:
        rate, dt, cores, E_o = cpu_oracle_iteration_rate(wl, ORACLE_ITERS, want_field=True)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{ORACLE_ITERS} FP64 oracle iterations from zero of the full {nx}x{ny}x{nz} grid "
                         f"({dt:.1f} s; scipy.fft workers = cores, NumPy elementwise on one core)"}
        parity = {"against": "FP64 oracle, equal iteration count from zero", "iterations": ORACLE_ITERS,
                  "field_rel_l2": float(np.linalg.norm(E_k - E_o) / np.linalg.norm(E_o)),
                  "field_max_abs_rel": float(np.abs(E_k - E_o).max() / np.abs(E_o).max())}
        del E_o
    sf, sa, obj = stats[-1]
    cfg = base_config(wl, args.tol)
    cfg.update({"iters_forward": sf.iters, "iters_adjoint": sa.iters, "rel_resid_forward": sf.rel_resid,
                "rel_resid_adjoint": sa.rel_resid, "objective": obj, "parallelism": f"replicas x{world}",
                "iteration_ms": iter_ms, "passes": pass_table, "check_every": args.check_every})
    plan.close()
    serving = None
    if args.serve_requests > 0 and args.tol > 0:
        # served-solve latency (the metric's third part), after the timed region: a seeded
        # stream of small grids through the continuous-batching server
        from paper_2506_15411_gb300 import inputs as _in
        from paper_2506_15411_gb300.serve import measure_stream
        serving = measure_stream(args.serve_requests, [_in.parse_size(v) for v in args.serve_sizes],
                                 tol=args.tol)
    if cufft is not None:
        cufft["ours_ms_per_iteration"] = iter_ms
        cufft["speedup_of_fused_kernels"] = cufft["ms_per_iteration"] / iter_ms
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
            "gpu_launches": launches * world, "clocks": clocks, "serving": serving,
            "cufft_comparison": cufft}
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


def load_traffic(kernel):
    """DRAM bytes per launch of `kernel` on this workload from the committed ncu summary
    (profiles/traffic_fresnel_lens_275x275x315.json), or None when the kernels have changed
    since those counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic_fresnel_lens_275x275x315.json")
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
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--max-iter", type=int, default=200000)
    ap.add_argument("--check-every", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=12,
                    help="requests of the served-latency stream after the timed region (0: none; "
                         "skipped when --tol <= 0)")
    ap.add_argument("--serve-sizes", nargs="+", default=["64", "128"], help="grid sizes of that stream")
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
