// stockham.cuh -- block-cooperative mixed-radix Stockham FFT over columns held in shared
// memory, with fused loaders and storers at the two ends.
//
// Stage q (radix R, Ns = product of the earlier radices) maps butterfly j (0 <= j < n/R):
//   inputs   x[j + r n/R],                          r = 0..R-1
//   twiddle  x_r *= w_n^{(j mod Ns) r n / (Ns R)}   (w_n = exp(-2 pi i / n); conj for inverse)
//   DFT_R in registers
//   outputs  y[(j - j mod Ns) R + j mod Ns + r Ns]
// and the last stage leaves the transform in natural order (self-sorting).  The first stage
// reads positions j + r n/R and the last writes positions j + r n/R, so for data in global
// memory both are coalesced when consecutive threads take consecutive j (x passes) or
// consecutive columns (y and z passes).  A stage holds one butterfly of one component per
// thread in registers (R values); a transform is run by T = n / min(R) threads.  Per-stage
// constants (R, Ns, n/R, twiddle step) come precomputed from a small device table.
#pragma once
#include "cbs_internal.h"
#include "fft_radix.cuh"

namespace cbs {

// This thread's column in shared memory: element i of component c at buf[c * sc + i * si].
struct SCol {
  float2* buf;
  int si;
  int sc;
  __device__ __forceinline__ float2& at(int c, int i) const { return buf[c * sc + i * si]; }
};

constexpr int kMaxRadix = 16;

template <int R, bool INV>
__device__ __forceinline__ void twiddle_dft(float2* v, int j, int Ns, int twstep,
                                            const float2* __restrict__ tw) {
  if constexpr (R > 1) {
    if (Ns > 1) {
      const int step = (j % Ns) * twstep;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = __ldg(&tw[r * step]);
        if (INV) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
  }
  DFT<R, INV>::run(v);
}

// Stage 0 from global memory: ld(c, i) returns component c at position i; the outputs of
// components c0..c1-1 go to shared memory (no barrier inside; the caller synchronises).
template <int R, bool INV, class Load>
__device__ __forceinline__ void stage_first_g(Load& ld, SCol s, int c0, int c1, int stride, int j,
                                              bool act) {
  if (!act) return;
  for (int c = c0; c < c1; ++c) {
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ld(c, j + r * stride);
    DFT<R, INV>::run(v);
#pragma unroll
    for (int r = 0; r < R; ++r) s.at(c, j * R + r) = v[r];
  }
}

// In-place stage in shared memory for component c: read, barrier, write, barrier.  With
// Ns = 1 it is a first stage whose input already sits in shared memory.  The barriers sit
// outside the radix switch and the butterfly lives in one register array of kMaxRadix
// slots, so the values of different radices are never live at the same time.
template <bool INV>
__device__ __forceinline__ void stage_mid(int R, SCol s, int c, int stride, int Ns, int twstep, int j,
                                          bool act, const float2* __restrict__ tw) {
  float2 v[kMaxRadix];
  if (act) {
    radix_dispatch(R, [&](auto Ri) {
      constexpr int RR = decltype(Ri)::value;
#pragma unroll
      for (int r = 0; r < RR; ++r) v[r] = s.at(c, j + r * stride);
      twiddle_dft<RR, INV>(v, j, Ns, twstep, tw);
    });
  }
  __syncthreads();
  if (act) {
    const int k = j % Ns;
    const int d = (j - k) * R + k;
    radix_dispatch(R, [&](auto Ri) {
      constexpr int RR = decltype(Ri)::value;
#pragma unroll
      for (int r = 0; r < RR; ++r) s.at(c, d + r * Ns) = v[r];
    });
  }
  __syncthreads();
}

// Last stage (Ns = n/R, so the outputs sit at j + r Ns): shared memory -> st(c, i, value).
template <int R, bool INV, class Store>
__device__ __forceinline__ void stage_last_g(Store& st, SCol s, int c0, int c1, int stride, int Ns,
                                             int twstep, int j, bool act,
                                             const float2* __restrict__ tw) {
  if (!act) return;
  for (int c = c0; c < c1; ++c) {
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s.at(c, j + r * stride);
    twiddle_dft<R, INV>(v, j, Ns, twstep, tw);
#pragma unroll
    for (int r = 0; r < R; ++r) st(c, j + r * Ns, v[r]);
  }
}

// Last stage written back to the same shared-memory positions it read (no barrier needed:
// each thread overwrites only its own inputs).
template <int R, bool INV>
__device__ __forceinline__ void stage_last_s(SCol s, int c, int stride, int Ns, int twstep, int j,
                                             bool act, const float2* __restrict__ tw) {
  if (!act) return;
  float2 v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = s.at(c, j + r * stride);
  twiddle_dft<R, INV>(v, j, Ns, twstep, tw);
#pragma unroll
  for (int r = 0; r < R; ++r) s.at(c, j + r * stride) = v[r];
}

// Single-stage transform (n == R): global -> registers -> global.
template <int R, bool INV, class Load, class Store>
__device__ __forceinline__ void stage_only_g(Load& ld, Store& st, int c0, int c1, bool act) {
  if (!act) return;
  for (int c = c0; c < c1; ++c) {
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ld(c, r);
    DFT<R, INV>::run(v);
#pragma unroll
    for (int r = 0; r < R; ++r) st(c, r, v[r]);
  }
}

// Stage q of a plan: {r, Ns, stride, twstep}.
__device__ __forceinline__ int4 stage_of(const AxisPlan& ap, int q) { return __ldg(&ap.st[q]); }

// Whole transform of components [0, nc) of this thread's column: global -> global through
// shared memory.  Every thread of the block must call it (barriers); col_ok masks the work.
template <bool INV, class Load, class Store>
__device__ __forceinline__ void fft_columns(const AxisPlan& ap, int nc, Load& ld, Store& st, SCol s,
                                            int t, bool col_ok, const float2* __restrict__ tw) {
  const int ns = ap.ns;
  if (ns == 1) {
    const int4 g = stage_of(ap, 0);
    radix_dispatch(g.x, [&](auto Ri) {
      constexpr int R = decltype(Ri)::value;
      stage_only_g<R, INV>(ld, st, 0, nc, col_ok && t == 0);
    });
    return;
  }
  {
    const int4 g = stage_of(ap, 0);
    radix_dispatch(g.x, [&](auto Ri) {
      constexpr int R = decltype(Ri)::value;
      stage_first_g<R, INV>(ld, s, 0, nc, g.z, t, col_ok && t < g.z);
    });
  }
  __syncthreads();
  for (int c = 0; c < nc; ++c) {
    for (int q = 1; q < ns - 1; ++q) {
      const int4 g = stage_of(ap, q);
      stage_mid<INV>(g.x, s, c, g.z, g.y, g.w, t, col_ok && t < g.z, tw);
    }
  }
  const int4 g = stage_of(ap, ns - 1);
  radix_dispatch(g.x, [&](auto Ri) {
    constexpr int R = decltype(Ri)::value;
    stage_last_g<R, INV>(st, s, 0, nc, g.z, g.y, g.w, t, col_ok && t < g.z, tw);
  });
}

}  // namespace cbs
