"""Host-side helpers on the CPU: FFT-friendly sizes of the resolution sweep, grid-size parsing,
latency percentiles, and the rule that bench.py reports ncu DRAM traffic only for the kernel
sources it was measured on."""
from __future__ import annotations

import json

import numpy as np

import bench
from paper_2506_15411_gb300 import inputs, sweep
from paper_2506_15411_gb300.serve import percentile


def test_fft_sizes_and_the_sweep_grid():
    for n in (1, 2, 13, 26, 275, 315, 640, 1001):
        assert sweep.fft_size(n) == n
    assert sweep.fft_size(17) == 18 and sweep.fft_size(289) == 294 and sweep.fft_size(323) == 324
    for m in range(1, 400):
        k = sweep.fft_size(m)
        assert k >= m
        r = k
        for p in (2, 3, 5, 7, 11, 13):
            while r % p == 0:
                r //= p
        assert r == 1
    nx, ny, nz, pitch, pads = sweep.grid_for(16)
    assert (nx, ny, nz) == (275, 275, 315) and pads == (16, 16, 96)   # the lens workload's grid


def test_parse_size_and_percentiles():
    assert inputs.parse_size("64") == (64, 64, 64)
    assert inputs.parse_size("192x192x128") == (192, 192, 128)
    x = list(range(1, 101))
    assert percentile(x, 50) == float(np.percentile(x, 50)) and percentile([], 50) != percentile([], 50)


def test_traffic_is_reported_only_for_the_measured_sources(tmp_path, monkeypatch):
    rec = {"source_sha256": bench.source_digest(), "bytes_per_launch": {"k_zpass_green": 123}}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "source_digest", lambda: rec["source_sha256"])
    assert bench.load_traffic("k_zpass_green", str(path)) == 123.0
    assert bench.load_traffic("k_ypass_fwd", str(path)) is None
    monkeypatch.setattr(bench, "source_digest", lambda: "0" * 64)     # sources changed since
    assert bench.load_traffic("k_zpass_green", str(path)) is None
    assert bench.load_traffic("k_zpass_green", str(tmp_path / "missing.json")) is None
