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


def test_wall_clock_limit_ends_a_solve_with_its_last_iterate():
    """A limit that runs out stops the series at a block boundary with CBS_ERR_TIME_LIMIT and
    the last iterate in E (equal to a plain run of the same number of iterations); a limit
    that does not run out leaves the result unchanged."""
    import torch
    from paper_2506_15411_gb300 import CBSPlan, PlaneWave
    from paper_2506_15411_gb300 import _lib as L
    n = 64
    eps = torch.from_numpy(inputs.random_eps(n, n, n, seed=4)).cuda()
    with CBSPlan(n, n, n, LAM / 8, LAM, 1.0, (8,) * 3, (8,) * 3, tol=1e-12, max_iter=1_000_000,
                 check_every=16) as plan:
        plan.set_permittivity(eps)
        plan.set_time_limit(0.05)
        E, s = plan.forward(PlaneWave())
        torch.cuda.synchronize()
        assert s.status == L.CBS_ERR_TIME_LIMIT and not s.converged
        assert 16 <= s.iters < 1_000_000 and s.iters % 16 == 0 and 0.05 <= s.seconds < 5.0
        assert np.isfinite(E.abs().max().item())
        plan.set_time_limit(0.0)
        plan.set_solver(0.0, s.iters, 16)
        E2, s2 = plan.forward(PlaneWave())
        plan.set_time_limit(600.0)
        E3, s3 = plan.forward(PlaneWave())
        torch.cuda.synchronize()
    assert s2.status == L.CBS_OK and s2.iters == s.iters and torch.equal(E, E2)
    assert s3.status == L.CBS_OK and s3.iters == s.iters and torch.equal(E2, E3)
    with pytest.raises(L.CBSError):
        with CBSPlan(n, n, n, LAM / 8, LAM, 1.0, (8,) * 3, (8,) * 3) as plan:
            plan.set_time_limit(-1.0)


def test_non_finite_source_ends_the_solve_as_diverged_and_the_plan_recovers():
    """A user source holding a NaN (made on the host; no GPU fault) makes the residual
    non-finite: the solve returns CBS_ERR_DIVERGED at the first check, and the next solve on
    the same plan with a finite source runs normally."""
    import torch
    from paper_2506_15411_gb300 import CBSPlan, PlaneWave, UserSource
    from paper_2506_15411_gb300 import _lib as L
    nx, ny, nz = 24, 20, 16
    eps = torch.from_numpy(inputs.random_eps(nx, ny, nz, seed=3)).cuda()
    S = torch.zeros((3, nz, ny, nx), dtype=torch.complex64)
    S[0, nz // 2, ny // 2, nx // 2] = complex(float("nan"), 0.0)
    S = S.cuda()
    with CBSPlan(nx, ny, nz, LAM / 8, LAM, 1.0, (3, 3, 3), (3, 3, 3), tol=1e-6, max_iter=64,
                 check_every=8) as plan:
        plan.set_permittivity(eps)
        with pytest.raises(L.CBSError) as ei:
            plan.forward(UserSource(S))
        assert ei.value.code == L.CBS_ERR_DIVERGED and "diverged" in str(ei.value)
        plan.set_solver(0.0, 16, 8)
        E, s = plan.forward(PlaneWave())
        torch.cuda.synchronize()
    assert s.status == L.CBS_OK and s.iters == 16 and torch.isfinite(torch.view_as_real(E)).all()
