"""GPU: the continuous-batching server (cbs_server_*).

* every result is bit-for-bit the same alone (one request on the GPU at a time) and in a mix
  of requests of different shapes admitted together;
* a served solve equals the same solve through a plan, and a served request of fixed length
  (tol 0) matches the FP64 oracle element by element: field, adjoint-driven gradient and
  objective;
* admission never holds more device memory than the budget, and a request that can never
  fit ends with CBS_ERR_OOM instead of waiting;
* requests are admitted while others run (no more than max_active at a time) and their work
  overlaps;
* same-shape requests in flight share the launches of their iterations.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import cbs_oracle as co
from paper_2506_15411_gb300 import inputs

pytestmark = pytest.mark.gpu

SIZES = ((32, 32, 32), (48, 40, 36), (64, 64, 64))


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("CUDA is not available: GPU tests need a GPU")
    return torch


def _stream(n, seed=5):
    from paper_2506_15411_gb300.serve import stream_request
    return [stream_request(rq) for rq in inputs.serving_stream(n, SIZES, seed=seed, ppl=8)]


def _submit(srv, rq):
    return srv.submit(rq["grid"], inputs.request_eps(rq), rq["source"], rq["r0"], adjoint=rq["adjoint"],
                      want_field=True, want_grad=rq["adjoint"], tag=rq["index"])


def test_results_are_identical_alone_and_in_the_mix():
    torch = _torch()
    from paper_2506_15411_gb300.serve import Server
    reqs = _stream(8)
    assert len({rq["grid"] for rq in reqs}) >= 2 and any(rq["adjoint"] for rq in reqs)
    alone = {}
    with Server(max_active=1, tol=1e-4, check_every=16) as srv:
        for rq in reqs:
            _submit(srv, rq)
            r = srv.wait(1)[0]
            alone[r.tag] = r
    with Server(max_active=8, tol=1e-4, check_every=16) as srv:
        for rq in reqs:
            _submit(srv, rq)
        mix = {r.tag: r for r in srv.wait(len(reqs))}
    torch.cuda.synchronize()
    for rq in reqs:
        a, b = alone[rq["index"]], mix[rq["index"]]
        assert a.ok and b.ok, (a.error, b.error)
        assert a.fwd.iters == b.fwd.iters and a.adj.iters == b.adj.iters
        assert a.objective == b.objective
        assert torch.equal(a.E, b.E)
        if rq["adjoint"]:
            assert a.adj.iters > 0 and torch.equal(a.grad, b.grad)


def test_served_solve_equals_the_plan_path():
    torch = _torch()
    from paper_2506_15411_gb300 import CBSPlan
    from paper_2506_15411_gb300.serve import Server
    rq = [q for q in _stream(8) if q["adjoint"]][0]
    g = rq["grid"]
    eps = inputs.request_eps(rq)
    with Server(max_active=2, tol=1e-4, check_every=16) as srv:
        _submit(srv, rq)
        r = srv.wait(1)[0]
    with CBSPlan(g.nx, g.ny, g.nz, g.pitch, g.lam, g.n_bg, g.pad_lo, g.pad_hi, tol=1e-4, check_every=16) as plan:
        plan.set_permittivity(torch.from_numpy(eps).cuda())
        E, st = plan.forward(rq["source"])
        Ea, sa = plan.adjoint(rq["r0"], E)
        grad, obj = plan.gradient(E, Ea, rq["r0"])
        torch.cuda.synchronize()
    assert r.ok and st.converged and sa.converged
    assert r.fwd.iters == st.iters and r.adj.iters == sa.iters
    assert r.objective == obj
    assert torch.equal(r.E, E) and torch.equal(r.grad, grad)


def test_served_request_matches_the_oracle_at_fixed_iterations():
    torch = _torch()
    from paper_2506_15411_gb300.serve import Server
    K = 200
    rq = [q for q in _stream(8) if q["adjoint"] and q["grid"].nx == 32][0]
    g = rq["grid"]
    eps = inputs.request_eps(rq)
    with Server(max_active=2, tol=0.0, max_iter=K, check_every=50) as srv:
        _submit(srv, rq)
        r = srv.wait(1)[0]
    torch.cuda.synchronize()
    assert r.ok, r.error      # tol 0: exactly K iterations each, no stopping rule applies
    assert r.fwd.iters == K and r.adj.iters == K
    og = co.Grid(g.nx, g.ny, g.nz, g.pitch, g.lam, g.n_bg, g.pad_lo, g.pad_hi)
    fwd = co.forward(og, eps.astype(np.float64), co.plane_wave_source(og, pol=rq["pol"]), tol=0.0, max_iter=K)
    adj = co.adjoint(og, eps.astype(np.float64), fwd.E, rq["r0"], tol=0.0, max_iter=K)
    grad = co.gradient(og, fwd.E, adj.E)
    obj = co.objective(fwd.E, rq["r0"])
    E = r.E.cpu().numpy()
    assert np.linalg.norm(E - fwd.E) <= 2e-5 * np.linalg.norm(fwd.E)
    gg = r.grad.cpu().numpy()
    assert np.linalg.norm(gg - grad) <= 1e-4 * np.linalg.norm(grad)
    assert abs(r.objective - obj) <= 1e-5 * obj
    assert abs(r.fwd.rel_resid - fwd.rel_resid) <= 1e-3 * fwd.rel_resid


def test_admission_stays_within_the_memory_budget():
    torch = _torch()
    from paper_2506_15411_gb300._lib import CBS_ERR_OOM
    from paper_2506_15411_gb300.serve import Server
    reqs = _stream(10, seed=9)
    big = max(rq["grid"].nx * rq["grid"].ny * rq["grid"].nz for rq in reqs)
    budget = 2.0 * big * 140 / 1e9 + 0.04     # room for about two of the largest slots
    with Server(max_active=8, hbm_budget_gb=budget, tol=1e-3, check_every=16) as srv:
        for rq in reqs:
            _submit(srv, rq)
        peak = 0.0
        got = []
        while len(got) < len(reqs):
            got += srv.take(64, 0.01)
            peak = max(peak, srv.info()["bytes_used"])
        assert all(r.ok for r in got)
        assert 0 < peak <= budget * 1e9
        # a grid whose slot alone is over the budget fails instead of waiting
        huge = dict(reqs[0], grid=type(reqs[0]["grid"])(256, 256, 256, reqs[0]["grid"].pitch, reqs[0]["grid"].lam,
                                                          1.0, (8, 8, 8), (8, 8, 8)))
        srv.submit(huge["grid"], np.ones((256, 256, 256), np.float32), huge["source"], (128, 128, 128))
        r = srv.wait(1)[0]
        assert r.status == CBS_ERR_OOM and "budget" in r.error
    torch.cuda.synchronize()


def test_requests_are_admitted_while_others_run():
    torch = _torch()
    from paper_2506_15411_gb300.serve import Server
    reqs = [q for q in _stream(24, seed=11) if q["grid"].nx == 64][:6]
    assert len(reqs) == 6
    with Server(max_active=3, tol=1e-4, check_every=16) as srv:
        for rq in reqs:
            srv.submit(rq["grid"], inputs.request_eps(rq), rq["source"], rq["r0"], adjoint=rq["adjoint"])
        res = srv.wait(len(reqs))
    torch.cuda.synchronize()
    assert all(r.ok for r in res)
    # never more than max_active admitted at once
    for r in res:
        running = sum(1 for q in res if q.t_admit <= r.t_admit < q.t_done)
        assert running <= 3
    # the first three run together; the others start as slots free up, before all are done
    first = sorted(res, key=lambda r: r.t_admit)
    assert first[1].t_admit < first[0].t_done and first[2].t_admit < first[0].t_done
    later = first[3:]
    assert all(r.t_admit >= min(q.t_done for q in first[:3]) - 1e-3 for r in later)
    assert min(r.t_admit for r in later) < max(q.t_done for q in first[:3])


def test_a_large_request_is_not_starved_by_a_stream_of_small_ones():
    """With memory for the large request only while no small slot is held, later small
    requests may pass it a bounded number of times (8); then admission waits for it."""
    torch = _torch()
    from paper_2506_15411_gb300 import PlaneWave
    from paper_2506_15411_gb300.serve import GridSpec, Server
    lam = 1.064e-6
    small = GridSpec(32, 32, 32, lam / 8, lam, 1.0, (4, 4, 4), (4, 4, 4))
    large = GridSpec(64, 64, 64, lam / 8, lam, 1.0, (8, 8, 8), (8, 8, 8))

    def slot_bytes(g):   # the server's footprint of a one-seat batch: the plan's arrays at
        nxp = (g.nx + 15) // 16 * 16   # padded rows, eps, E, E_adj, gradient, 16 MB of tables
        return nxp * g.ny * g.nz * 56 + g.nx * g.ny * g.nz * 56 + (16 << 20)

    budget = (slot_bytes(large) + (1 << 20)) / 1e9
    eps_s = inputs.random_eps(32, 32, 32, seed=21)
    eps_l = inputs.random_eps(64, 64, 64, seed=22)
    with Server(max_active=4, hbm_budget_gb=budget, tol=1e-3, check_every=16) as srv:
        for i in range(2):
            srv.submit(small, eps_s, PlaneWave(), (16, 16, 20), tag=("s", i))
        srv.submit(large, eps_l, PlaneWave(), (32, 32, 40), tag=("L", 0))
        for i in range(2, 26):
            srv.submit(small, eps_s, PlaneWave(), (16, 16, 20), tag=("s", i))
        res = {r.tag: r for r in srv.wait(26 + 1)}
    torch.cuda.synchronize()
    assert all(r.ok for r in res.values()), [r.error for r in res.values() if not r.ok]
    big = res[("L", 0)]
    passed = sum(1 for i in range(2, 26) if res[("s", i)].t_admit < big.t_admit)
    assert passed <= 8, passed
    assert big.fwd.iters > 0


def test_same_shape_requests_share_launches():
    """Four same-shape requests admitted together run in one batch: launches carry several of
    them, and each result equals the one it gets alone."""
    torch = _torch()
    from paper_2506_15411_gb300.serve import Server
    reqs = [q for q in _stream(24, seed=11) if q["grid"].nx == 32][:4]
    assert len(reqs) == 4
    alone = {}
    with Server(max_active=1, tol=1e-4, check_every=16) as srv:
        for rq in reqs:
            _submit(srv, rq)
            r = srv.wait(1)[0]
            alone[r.tag] = r
        sh1 = srv.sharing()
    with Server(max_active=4, tol=1e-4, check_every=16) as srv:
        for rq in reqs:
            _submit(srv, rq)
        mix = {r.tag: r for r in srv.wait(len(reqs))}
        sh = srv.sharing()
    torch.cuda.synchronize()
    assert sh1["max_members"] == 1 and sh1["request_iterations"] == sh1["launches"]
    assert sh["max_members"] >= 2, sh
    total = sum(r.fwd.iters + r.adj.iters for r in mix.values())
    assert sh["request_iterations"] == total, (sh, total)
    assert sh["launches"] < sh["request_iterations"], sh
    for rq in reqs:
        a, b = alone[rq["index"]], mix[rq["index"]]
        assert a.ok and b.ok, (a.error, b.error)
        assert a.fwd.iters == b.fwd.iters and a.adj.iters == b.adj.iters
        assert torch.equal(a.E, b.E)
        if rq["adjoint"]:
            assert torch.equal(a.grad, b.grad)


def test_requests_share_launches_only_with_the_same_plan_settings():
    """Same grid, different absorbing layers: separate batches (a launch never mixes plans);
    the same layers: one batch.  Each result equals the plan path with its own layers."""
    torch = _torch()
    import dataclasses
    from paper_2506_15411_gb300 import CBSPlan
    from paper_2506_15411_gb300.serve import Server
    rq = [q for q in _stream(24, seed=11) if q["grid"].nx == 32][0]
    g0 = rq["grid"]
    g1 = dataclasses.replace(g0, layer_round_trip=1e-2, layer_corner_max=True)
    eps = inputs.request_eps(rq)
    res = {}
    for tag, grids in (("mixed", (g0, g1)), ("same", (g1, g1))):
        with Server(max_active=2, tol=1e-4, check_every=16) as srv:
            for i, g in enumerate(grids):
                srv.submit(g, eps, rq["source"], rq["r0"], want_field=True, tag=i)
            out = {r.tag: r for r in srv.wait(2)}
            res[tag] = (out, srv.sharing())
    torch.cuda.synchronize()
    assert res["mixed"][1]["max_members"] == 1
    assert res["same"][1]["max_members"] == 2
    for g, r in ((g0, res["mixed"][0][0]), (g1, res["mixed"][0][1]), (g1, res["same"][0][0])):
        assert r.ok, r.error
        with CBSPlan(g.nx, g.ny, g.nz, g.pitch, g.lam, g.n_bg, g.pad_lo, g.pad_hi, tol=1e-4, check_every=16,
                     layer_round_trip=g.layer_round_trip, layer_corner_max=g.layer_corner_max) as plan:
            plan.set_permittivity(torch.from_numpy(eps).cuda())
            E, st = plan.forward(rq["source"])
            torch.cuda.synchronize()
        assert r.fwd.iters == st.iters and torch.equal(r.E, E)
    assert res["mixed"][0][1].fwd.iters != res["mixed"][0][0].fwd.iters or \
        not torch.equal(res["mixed"][0][1].E, res["mixed"][0][0].E)
