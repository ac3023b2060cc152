"""The multi-GPU path of bench.py is replicas only: each rank solves its own problem and the
ranks meet once, after the timed region, to take the slowest time and the total work.  That
combination runs here as two gloo ranks on the CPU (no GPU, no collective on the data path)."""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r timed (10 + r, 20 - r) ms over (100 (r + 1), 7) iterations
        t, c = bench.combine_ranks([10.0 + rank, 20.0 - rank], [100.0 * (rank + 1), 7.0], world, torch.device("cpu"))
        q.put((rank, t, c))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_all_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, c in out:
        assert t == [11.0, 20.0] and c == [300.0, 14.0], (rank, t, c)


def test_one_rank_passes_its_numbers_through():
    import torch
    import bench
    assert bench.combine_ranks([3.0, 4.0], [5.0, 6.0], 1, torch.device("cpu")) == ([3.0, 4.0], [5.0, 6.0])
