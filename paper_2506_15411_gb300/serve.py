"""Serving: continuous batching of CBS solves over mixed grid sizes.

The server itself is native (cbs_server_* in include/cbs.h): a worker thread admits queued
requests into per-shape batches within a device-memory budget -- a batch iterates all of its
requests in the same launches -- and advances every batch one block of iterations at a time,
so new requests start while others run and batches of different shapes share the GPU.  This
module marshals requests and results, and drives a stream of timed arrivals for latency
measurements:

    python -m paper_2506_15411_gb300.serve --requests 40 --sizes 64 128 192x192x128 --layers gentle

prints one JSON line: p50 / p99 latency, solves/s, and the single-solve times of the same
requests run alone.
"""
from __future__ import annotations

import ctypes
import threading
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L
from .solver import PlaneWave, PointSource, Stats, _stats


@dataclass(frozen=True)
class GridSpec:
    nx: int
    ny: int
    nz: int
    pitch: float
    lam: float
    n_bg: float = 1.0
    pad_lo: tuple = (0, 0, 0)
    pad_hi: tuple = (0, 0, 0)
    layer_round_trip: float = 0.0    # absorbing layers as in CBSPlan (0: defaults)
    layer_power: float = 0.0
    layer_corner_max: bool = False

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


@dataclass
class Result:
    id: int
    status: int
    objective: float
    fwd: Stats
    adj: Stats
    t_submit: float
    t_admit: float
    t_done: float
    error: str
    E: Optional[torch.Tensor] = None
    grad: Optional[torch.Tensor] = None
    tag: object = None

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit

    @property
    def ok(self) -> bool:
        return self.status == L.CBS_OK


def _source_struct(src) -> L.cbs_source:
    s = L.cbs_source()
    s.z_plane = -1
    if isinstance(src, PlaneWave):
        s.kind = L.CBS_SRC_PLANE_WAVE
        s.z_plane = src.z_plane
    elif isinstance(src, PointSource):
        s.kind = L.CBS_SRC_POINT
        for i in range(3):
            s.r0[i] = int(src.r0[i])
    else:
        raise TypeError("served solves take PlaneWave or PointSource sources")
    for i in range(3):
        p = complex(src.pol[i])
        s.pol[i][0] = p.real
        s.pol[i][1] = p.imag
    return s


class Server:
    """A continuous-batching CBS server on the current CUDA device."""

    def __init__(self, max_active: int = 8, hbm_budget_gb: float = 0.0, tol: float = 1e-4,
                 max_iter: int = 100000, check_every: int = 32):
        self.lib = L.lib()
        d = L.cbs_server_desc(float(hbm_budget_gb) * 1e9, int(max_active), float(tol), int(max_iter),
                              int(check_every))
        h = ctypes.c_void_p()
        L.check(self.lib.cbs_server_create(ctypes.byref(h), ctypes.byref(d)))
        self.handle = h
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._keep: Dict[int, tuple] = {}
        self._buf = (L.cbs_result * 64)()

    def close(self):
        if getattr(self, "handle", None):
            self.lib.cbs_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, grid: GridSpec, eps, source, r0, adjoint: bool = False, want_field: bool = False,
               want_grad: bool = False, field_on_device: bool = True, tag=None) -> int:
        """Queue one solve.  eps: float32 (nz, ny, nx), a numpy array (copied at admission) or
        a CUDA tensor.  want_field / want_grad: return E (complex64 (3, nz, ny, nx)) / dL/d eps
        on the device (field_on_device) or in pinned host memory."""
        r = L.cbs_request()
        r.nx, r.ny, r.nz = grid.nx, grid.ny, grid.nz
        r.pitch_m, r.lambda_m, r.n_bg = grid.pitch, grid.lam, grid.n_bg
        for i in range(3):
            r.pad_lo[i] = int(grid.pad_lo[i])
            r.pad_hi[i] = int(grid.pad_hi[i])
            r.r0[i] = int(r0[i])
        r.layer_round_trip = float(grid.layer_round_trip)
        r.layer_power = float(grid.layer_power)
        r.layer_corner_max = 1 if grid.layer_corner_max else 0
        if isinstance(eps, torch.Tensor):
            if eps.dtype != torch.float32 or not eps.is_cuda or not eps.is_contiguous() or tuple(eps.shape) != grid.shape:
                raise ValueError("eps must be a contiguous float32 CUDA tensor of the grid's shape")
            r.eps_dev = eps.data_ptr()
        else:
            eps = np.ascontiguousarray(eps, dtype=np.float32)
            if eps.shape != grid.shape:
                raise ValueError("eps shape")
            r.eps_host = eps.ctypes.data
        r.src = _source_struct(source)
        r.adjoint = 1 if adjoint else 0
        E = g = None
        if want_field:
            shape = (3,) + grid.shape
            E = torch.empty(shape, dtype=torch.complex64, device=self.device) if field_on_device else \
                torch.empty(shape, dtype=torch.complex64, pin_memory=True)
            if field_on_device:
                r.E_dev = E.data_ptr()
            else:
                r.E_host = E.data_ptr()
        if want_grad:
            if not adjoint:
                raise ValueError("want_grad needs adjoint=True")
            g = torch.empty(grid.shape, dtype=torch.float32, device=self.device) if field_on_device else \
                torch.empty(grid.shape, dtype=torch.float32, pin_memory=True)
            if field_on_device:
                r.grad_dev = g.data_ptr()
            else:
                r.grad_host = g.data_ptr()
        rid = ctypes.c_longlong()
        L.check(self.lib.cbs_server_submit(self.handle, ctypes.byref(r), ctypes.byref(rid)))
        self._keep[rid.value] = (eps, E, g, tag)
        return rid.value

    def take(self, max_n: int = 64, timeout: float = 1.0) -> List[Result]:
        """Completed results (up to max_n), waiting up to `timeout` s for the first."""
        n = ctypes.c_int()
        L.check(self.lib.cbs_server_take(self.handle, self._buf, min(max_n, 64), float(timeout), ctypes.byref(n)))
        out = []
        for i in range(n.value):
            c = self._buf[i]
            _, E, g, tag = self._keep.pop(c.id, (None, None, None, None))
            out.append(Result(c.id, c.status, c.objective, _stats(c.fwd), _stats(c.adj), c.t_submit, c.t_admit,
                              c.t_done, c.error.decode(errors="replace"), E, g, tag))
        return out

    def wait(self, count: int, timeout: float = 3600.0) -> List[Result]:
        """Take `count` results, waiting up to `timeout` s in all."""
        out: List[Result] = []
        t_end = time.monotonic() + timeout
        while len(out) < count:
            left = t_end - time.monotonic()
            if left <= 0:
                raise TimeoutError(f"{len(out)} of {count} results after {timeout} s")
            out += self.take(64, min(left, 1.0))
        return out

    def info(self):
        q, a, b = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_double()
        L.check(self.lib.cbs_server_info(self.handle, ctypes.byref(q), ctypes.byref(a), ctypes.byref(b)))
        return {"queued": q.value, "active": a.value, "bytes_used": b.value}

    def sharing(self):
        """Launch sharing so far: iteration launches, request iterations they carried, and the
        most requests one launch carried."""
        n, m, mx = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int()
        L.check(self.lib.cbs_server_sharing(self.handle, ctypes.byref(n), ctypes.byref(m), ctypes.byref(mx)))
        return {"launches": n.value, "request_iterations": m.value, "max_members": mx.value}


# ------------------------------------------------------------------ timed request streams
@dataclass
class StreamReport:
    results: List[Result]
    p50_s: float
    p99_s: float
    mean_s: float
    solves_per_s: float
    makespan_s: float
    peak_active: int = 0
    extra: dict = field(default_factory=dict)


def percentile(x: Sequence[float], q: float) -> float:
    return float(np.percentile(np.asarray(x, dtype=np.float64), q)) if len(x) else float("nan")


def run_stream(server: Server, requests: Sequence[dict], make_eps, speed: float = 1.0) -> StreamReport:
    """Submit `requests` (dicts with grid, source, r0, adjoint, arrival_s) at their arrival
    times (divided by `speed`) and collect every result.  make_eps(request) builds the
    permittivity; a helper thread builds them ahead of their arrivals."""
    import queue as _q
    ready: "_q.Queue" = _q.Queue(maxsize=8)

    def producer():
        for rq in requests:
            ready.put((rq, make_eps(rq)))

    th = threading.Thread(target=producer, daemon=True)
    th.start()
    results: List[Result] = []
    peak = 0
    t0 = time.monotonic()
    for _ in range(len(requests)):
        rq, eps = ready.get()
        delay = t0 + rq["arrival_s"] / speed - time.monotonic()
        while delay > 0:
            results += server.take(64, min(delay, 0.05))
            delay = t0 + rq["arrival_s"] / speed - time.monotonic()
        server.submit(rq["grid"], eps, rq["source"], rq["r0"], adjoint=rq["adjoint"], tag=rq.get("index"))
        peak = max(peak, server.info()["active"])
    while len(results) < len(requests):
        results += server.take(64, 1.0)
        peak = max(peak, server.info()["active"])
    th.join()
    lat = [r.latency for r in results]
    span = max(r.t_done for r in results) - min(r.t_submit for r in results)
    return StreamReport(results, percentile(lat, 50), percentile(lat, 99), float(np.mean(lat)),
                        len(results) / span if span > 0 else float("nan"), span, peak)


# Absorbing-layer settings of a stream: the defaults, or the gentler one (round trip 1e-2,
# the largest profile where layers overlap) that converges in about a fifth of the iterations
LAYERS = {"default": {}, "gentle": {"layer_round_trip": 1e-2, "layer_corner_max": True}}


def stream_request(rq: dict, layers: str = "default") -> dict:
    """A request of inputs.serving_stream as the grid / source / r0 this module submits."""
    g = GridSpec(rq["nx"], rq["ny"], rq["nz"], rq["pitch"], rq["lam"], 1.0, tuple(rq["pads"]), tuple(rq["pads"]),
                 **LAYERS[layers])
    return dict(rq, grid=g, source=PlaneWave(pol=rq["pol"]))


def measure_stream(requests: int, sizes, ppl: int = 8, load: float = 0.8, max_active: int = 8,
                   tol: float = 1e-4, seed: int = 42, layers: str = "default", log=None) -> dict:
    """Serve a seeded stream (inputs.serving_stream, every size equally often) at `load` times
    the single-solve service rate and report latency percentiles and throughput, next to the
    service times of the same requests solved alone, one at a time.  log(tag, request, result)
    sees every result."""
    from . import inputs
    reqs = [stream_request(rq, layers) for rq in inputs.serving_stream(requests, sizes, seed=seed, ppl=ppl,
                                                                       balanced=True)]
    alone = []
    with Server(max_active=1, tol=tol) as srv:
        for rq in reqs:
            srv.submit(rq["grid"], inputs.request_eps(rq), rq["source"], rq["r0"], adjoint=rq["adjoint"])
            r = srv.wait(1)[0]
            if log:
                log("alone", rq, r)
            alone.append(r.t_done - r.t_admit)
    rate = load / float(np.mean(alone))
    inputs.assign_arrivals(reqs, rate, seed=seed)
    with Server(max_active=max_active, tol=tol) as srv:
        rep = run_stream(srv, reqs, inputs.request_eps)
        sharing = srv.sharing()
    if log:
        for r in rep.results:
            log("stream", reqs[r.tag], r)
    by_size = {}
    for rq, r in zip(reqs, sorted(rep.results, key=lambda r: r.tag)):
        by_size.setdefault("x".join(map(str, (rq["nx"], rq["ny"], rq["nz"]))), []).append(r.latency)
    return {"requests": len(reqs), "sizes": [list(v) for v in sizes], "tol": tol, "layers": layers,
            "max_active": max_active, "arrival_rate_hz": rate, "offered_load": load,
            "p50_latency_s": rep.p50_s, "p99_latency_s": rep.p99_s, "mean_latency_s": rep.mean_s,
            "solves_per_s": rep.solves_per_s, "makespan_s": rep.makespan_s, "peak_active": rep.peak_active,
            "single_solve_p50_s": percentile(alone, 50), "single_solve_p99_s": percentile(alone, 99),
            "single_solve_total_s": float(np.sum(alone)),
            "p50_latency_s_by_size": {k: percentile(v, 50) for k, v in by_size.items()},
            "requests_by_size": {k: len(v) for k, v in by_size.items()},
            "launches": sharing["launches"], "request_iterations": sharing["request_iterations"],
            "max_requests_per_launch": sharing["max_members"],
            "failed": sum(1 for r in rep.results if not r.ok)}


def main():
    import argparse
    import json
    import sys

    from . import inputs

    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=40)
    ap.add_argument("--sizes", nargs="+", default=["64", "128", "192x192x128"],
                    help="grid sizes: N for N^3 or NXxNYxNZ")
    ap.add_argument("--ppl", type=int, default=8)
    ap.add_argument("--load", type=float, default=0.8, help="offered load against single-solve service time")
    ap.add_argument("--max-active", type=int, default=8)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--seed", type=int, default=42)
    ap.add_argument("--layers", choices=sorted(LAYERS), default="default", help="absorbing-layer setting")
    ap.add_argument("--verbose", action="store_true", help="one line per result on stderr")
    args = ap.parse_args()

    def log(tag, rq, r):
        if args.verbose:
            print(json.dumps({"phase": tag, "grid": [rq["nx"], rq["ny"], rq["nz"]], "adjoint": rq["adjoint"],
                              "structure": rq["structure"], "status": r.status, "fwd_iters": r.fwd.iters,
                              "adj_iters": r.adj.iters, "service_s": r.t_done - r.t_admit,
                              "latency_s": r.latency}), file=sys.stderr, flush=True)

    sizes = [inputs.parse_size(v) for v in args.sizes]
    print(json.dumps(measure_stream(args.requests, sizes, args.ppl, args.load, args.max_active, args.tol,
                                    args.seed, args.layers, log)))


if __name__ == "__main__":
    main()
