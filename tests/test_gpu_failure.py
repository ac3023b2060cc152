"""GPU: the failure path of the tile kernels, without a GPU fault.  Their waits on tensor
copies are bounded; the self-test runs that bounded wait on an mbarrier nothing completes,
checks that it gives up with the timeout status, and that the context then still runs a solve."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_2506_15411_gb300 import inputs

pytestmark = pytest.mark.gpu

LAM = 1.064e-6


def test_bounded_wait_times_out_and_the_context_stays_usable():
    import torch
    from paper_2506_15411_gb300 import CBSPlan, PlaneWave
    from paper_2506_15411_gb300 import _lib as L
    torch.cuda.set_device(0)
    st = ctypes.c_int(-1)
    assert L.lib().cbs_selftest_wait_timeout(ctypes.byref(st)) == L.CBS_OK, L.lib().cbs_last_error()
    assert st.value == 1
    with CBSPlan(24, 20, 16, LAM / 8, LAM, 1.0, (3, 3, 3), (3, 3, 3), tol=0.0, max_iter=8, check_every=8) as plan:
        plan.set_permittivity(torch.from_numpy(inputs.random_eps(24, 20, 16, seed=2)).cuda())
        E, s = plan.forward(PlaneWave())
        torch.cuda.synchronize()
    assert s.iters == 8 and np.isfinite(E.abs().max().item())
