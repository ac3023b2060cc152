"""The in-place FFT stages of the CUDA library (csrc/fft_ip.cuh, csrc/axis_plan.h) run on the
CPU, one emulated thread at a time (tests/fft_host/fft_host.cu, built here with nvcc for the
host), against numpy.fft:

* forward (decimation in frequency) leaves frequency k at the position the wave-number table
  names, for column tiles (pairs and single columns, 1 and 3 components) and row tiles;
* inverse after forward (decimation in time) is n times the identity;
* the fused z stage (last forward stage, a pointwise multiply, first inverse stage) is the
  circular convolution n * IFFT(g * FFT(x));
* the fused x stage (last inverse stage, a pointwise map, first forward stage) gives the
  spectrum of the mapped natural-order values.
Lengths cover every radix, odd and even axes, one-stage axes, the workload axes (275, 315,
336, 640) and the longest ones (704, 1001, 1024); thread counts below and above the item counts.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fft_host", "fft_host.cu")
CSRC = os.path.join(os.path.dirname(HERE), "paper_2506_15411_gb300", "csrc")
LENGTHS = [1, 2, 3, 5, 7, 11, 13, 16, 30, 64, 105, 192, 275, 315, 336, 640, 704, 1001, 1024]
P = ctypes.c_void_p


@pytest.fixture(scope="module")
def fh(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("fft_host") / "libfft_host.so")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-Xcompiler", "-fPIC", "-shared", "--expt-relaxed-constexpr",
                    "-I", CSRC, "-o", out, SRC], check=True, capture_output=True)
    return ctypes.CDLL(out)


def _freq_of_pos(fh, n, layout, ncol):
    pq = np.zeros(2 * n, np.float32)
    assert fh.fh_pq(n, layout, ncol, pq.ctypes.data_as(P)) == 0
    pq = pq.reshape(n, 2)
    k = np.round(pq[:, 0] * n / (2 * np.pi)).astype(int) % n
    assert sorted(k) == list(range(n))               # a permutation of the frequencies
    nyq = (n % 2 == 0) & (k == n // 2)
    assert np.all(pq[nyq, 1] == 0) and np.all(pq[~nyq, 1] == pq[~nyq, 0])
    return k


def _cplx(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


@pytest.mark.parametrize("n", LENGTHS)
@pytest.mark.parametrize("layout,ncol,ncomp,pairs,nth",
                         [(1, 8, 1, 1, 512), (1, 16, 1, 0, 96), (2, 8, 3, 1, 512), (2, 4, 3, 1, 64)])
def test_column_stages_match_numpy(fh, n, layout, ncol, ncomp, pairs, nth):
    rng = np.random.default_rng(n)
    k = _freq_of_pos(fh, n, layout, ncol)
    x = _cplx(rng, (ncomp, n, ncol))
    spec, back = np.zeros_like(x), np.zeros_like(x)
    assert fh.fh_cols(n, layout, ncol, ncomp, nth, pairs, x.ctypes.data_as(P), spec.ctypes.data_as(P),
                      back.ctypes.data_as(P)) == 0
    X = np.fft.fft(x.astype(np.complex128), axis=1)
    scale = np.abs(X).max()
    assert np.abs(spec - X[:, k, :]).max() <= 2e-6 * scale
    assert np.abs(back - n * x).max() <= 2e-6 * n * np.abs(x).max()
    if layout == 2:
        p = 2 * np.pi * np.fft.fftfreq(n)
        g = (1.0 / (1.0 + p ** 2 + 0.3j)).astype(np.complex64)    # by frequency
        gpos = g[k]                                                  # by position
        out = np.zeros_like(x)
        assert fh.fh_zpass(n, ncol, nth, x.ctypes.data_as(P), gpos.ctypes.data_as(P), out.ctypes.data_as(P)) == 0
        want = n * np.fft.ifft(g[None, :, None].astype(np.complex128) * X, axis=1)
        assert np.abs(out - want).max() <= 2e-6 * np.abs(want).max()


@pytest.mark.parametrize("n", LENGTHS)
@pytest.mark.parametrize("nrows,nth", [(3, 512), (1, 40)])
def test_row_stages_and_the_fused_x_stage_match_numpy(fh, n, nrows, nth):
    rng = np.random.default_rng(1000 + n)
    k = _freq_of_pos(fh, n, 0, 0)
    ncomp, ld = 3, (n + 15) // 16 * 16
    x = _cplx(rng, (ncomp, nrows, ld))
    spec, back = np.zeros_like(x), np.zeros_like(x)
    assert fh.fh_rows(n, nrows, ncomp, ld, nth, x.ctypes.data_as(P), spec.ctypes.data_as(P),
                      back.ctypes.data_as(P)) == 0
    X = np.fft.fft(x[..., :n].astype(np.complex128), axis=2)
    assert np.abs(spec[..., :n] - X[..., k]).max() <= 2e-6 * np.abs(X).max()
    assert np.abs(back[..., :n] - n * x[..., :n]).max() <= 2e-6 * n * np.abs(x).max()
    a = _cplx(rng, (n,))
    b = _cplx(rng, (ncomp, nrows, ld))
    out = np.zeros_like(x)
    assert fh.fh_xpass(n, nrows, ncomp, ld, nth, spec.ctypes.data_as(P), a.ctypes.data_as(P),
                       b.ctypes.data_as(P), out.ctypes.data_as(P)) == 0
    u = a[None, None, :].astype(np.complex128) * (n * x[..., :n]) + b[..., :n]
    U = np.fft.fft(u, axis=2)
    assert np.abs(out[..., :n] - U[..., k]).max() <= 3e-6 * np.abs(U).max()


def test_radix_order_avoids_modelled_bank_conflicts(fh):
    """Row transforms end on a radix whose contiguous butterflies are conflict-free (odd, or
    2 mod 4 with 16-byte accesses); the C5 and C2 axes get the orders the model picks."""
    o = (ctypes.c_int * 8)()
    s = fh.fh_order(640, 0, 0, o)
    assert s == 3 and o[s - 1] % 4 != 0 and sorted(o[:s]) == [8, 8, 10]
    s = fh.fh_order(336, 2, 8, o)
    assert sorted(o[:s]) == [6, 7, 8]
    assert fh.fh_order(17, 0, 0, o) == -1          # not a product of the supported radices


def test_z_radix_order_balances_the_warp_groups_rounds(fh):
    """The z order puts the radix whose fused-stage items fill the 256-thread warp group best
    last: 315 = 5 7 9 would run the fused radix-9 stage in two rounds of 280 items (the second
    nearly idle), 5 9 7 in two rounds of 360; 336 keeps 8 6 7."""
    o = (ctypes.c_int * 8)()
    s = fh.fh_order_z(315, 8, 256, o)
    assert s == 3 and sorted(o[:s]) == [5, 7, 9] and o[s - 1] != 9
    s = fh.fh_order_z(336, 8, 256, o)
    assert list(o[:s]) == [8, 6, 7]
    assert fh.fh_order_z(17, 8, 256, o) == -1
    # the model by hand, 315 = 5 7 9 on 8-column tiles and 256 threads: stage 5 has 3 * 4 * 63
    # = 756 pair items (3 rounds x 2 directions x 2 * 5 values = 60), stage 7 has 540 (3 x 2 x
    # 14 = 84), the fused stage 9 has 8 * 35 = 280 single-column items (2 rounds x 6 * 9 = 108)
    fh.fh_z_balance.restype = ctypes.c_longlong
    assert fh.fh_z_balance(315, (ctypes.c_int * 3)(5, 7, 9), 3, 8, 256) == 252
    assert fh.fh_z_balance(315, (ctypes.c_int * 3)(5, 9, 7), 3, 8, 256) == 60 + 2 * 2 * 18 + 2 * 42
