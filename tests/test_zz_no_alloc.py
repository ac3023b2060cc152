"""The allocation-free splitting entry point (cbs_splitting_noalloc) against the plan path.

cbs_splitting_noalloc is for callers that cannot call cudaMalloc (their device memory is
owned by another allocator, or their loop must not synchronise on allocation).  It keeps its
block partial sums in one static device array that every call shares, so two calls in a row
on different grids also check that nothing stale from the first call leaks into the second.
This file is named so that pytest collects it last."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_2506_15411_gb300 import inputs

pytestmark = pytest.mark.gpu

LAM = 1.064e-6


def _desc(L, nx, ny, nz, pitch, lo, hi, stream=0, n_bg=1.0, rt=0.0, power=0.0, corner=0):
    return L.cbs_plan_desc(nx, ny, nz, pitch, LAM, n_bg, (ctypes.c_int * 3)(*lo), (ctypes.c_int * 3)(*hi),
                           0.0, 1, 1, ctypes.c_void_p(stream), rt, power, corner)


def _noalloc(L, lib, desc, eps):
    k0 = ctypes.c_double()
    ep = ctypes.c_double()
    rc = lib.cbs_splitting_noalloc(ctypes.byref(desc), ctypes.c_void_p(eps.data_ptr()), ctypes.byref(k0),
                                   ctypes.byref(ep))
    return rc, k0.value, ep.value


def test_noalloc_splitting_matches_plan_on_two_calls_in_a_row():
    import torch
    from paper_2506_15411_gb300 import CBSPlan
    from paper_2506_15411_gb300 import _lib as L
    lib = L.lib()
    # a large grid first (many block partials), then a small one that reuses fewer of them
    # (a third grid with a background index other than 1 checks the layer strength's n_bg, a
    # fourth the layer options)
    cases = [((96, 80, 110), LAM / 8, (8, 6, 10), (7, 8, 9), 1.0, 2.4, 31, 1.0, (0.0, 0.0, 0)),
             ((20, 18, 22), LAM / 6, (3, 2, 4), (2, 3, 1), 1.3, 1.6, 32, 1.0, (0.0, 0.0, 0)),
             ((40, 36, 30), LAM / 8, (4, 5, 6), (6, 5, 4), 1.7, 2.2, 34, 1.33, (0.0, 0.0, 0)),
             ((40, 36, 30), LAM / 8, (4, 5, 6), (6, 5, 4), 1.0, 2.2, 35, 1.0, (1e-2, 3.0, 1))]
    for (nx, ny, nz), pitch, lo, hi, emin, emax, seed, n_bg, (rt, pw, cm) in cases:
        eps = torch.from_numpy(inputs.random_eps(nx, ny, nz, lo=emin, hi=emax, seed=seed)).cuda()
        with CBSPlan(nx, ny, nz, pitch, LAM, n_bg, lo, hi, layer_round_trip=rt, layer_power=pw,
                     layer_corner_max=bool(cm)) as plan:
            plan.set_permittivity(eps)
            k0_ref, ep_ref = plan.splitting()
        torch.cuda.synchronize()
        rc, k0, ep = _noalloc(L, lib, _desc(L, nx, ny, nz, pitch, lo, hi, n_bg=n_bg, rt=rt, power=pw, corner=cm),
                              eps)
        assert rc == L.CBS_OK, lib.cbs_last_error()
        assert abs(k0 - k0_ref) <= 1e-12 * abs(k0_ref)
        assert abs(ep - ep_ref) <= 1e-12 * ep_ref


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    from paper_2506_15411_gb300 import _lib as L
    lib = L.lib()
    eps = torch.ones(8, dtype=torch.float32, device="cuda")   # never read: the size check comes first
    d = _desc(L, 1024, 1024, 257, LAM / 8, (0, 0, 0), (0, 0, 0))
    rc, _, _ = _noalloc(L, lib, d, eps)
    assert rc == L.CBS_ERR_ARG
    assert b"no-alloc limit" in lib.cbs_last_error()
    bad = torch.ones((6, 6, 6), dtype=torch.float32, device="cuda")
    bad[1, 2, 3] = float("inf")
    rc, _, _ = _noalloc(L, lib, _desc(L, 6, 6, 6, LAM / 8, (1, 1, 1), (1, 1, 1)), bad)
    assert rc == L.CBS_ERR_ARG and b"non-finite" in lib.cbs_last_error()
    # pads that cbs_plan rejects (over half the axis) are rejected here too
    from paper_2506_15411_gb300 import CBSPlan
    for lo, hi in (((4, 1, 1), (1, 1, 1)), ((1, 1, 1), (1, 1, 4))):
        with pytest.raises(L.CBSError):
            CBSPlan(7, 7, 7, LAM / 8, LAM, 1.0, lo, hi)
        rc, _, _ = _noalloc(L, lib, _desc(L, 7, 7, 7, LAM / 8, lo, hi), eps)
        assert rc == L.CBS_ERR_ARG and b"pads" in lib.cbs_last_error()
    # the scratch is still good after the rejected calls
    eps = torch.from_numpy(inputs.random_eps(12, 10, 14, seed=33)).cuda()
    rc, k0, ep = _noalloc(L, lib, _desc(L, 12, 10, 14, LAM / 8, (2, 2, 2), (2, 2, 2)), eps)
    assert rc == L.CBS_OK and ep > 0 and np.isfinite(k0)
