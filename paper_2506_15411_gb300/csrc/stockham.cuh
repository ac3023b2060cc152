// stockham.cuh -- block-cooperative mixed-radix Stockham FFT over tiles in shared memory.
//
// Stage q (radix R, Ns = product of the earlier radices) maps butterfly j (0 <= j < n/R):
//   inputs   x[j + r n/R],                          r = 0..R-1
//   twiddle  x_r *= w_n^{(j mod Ns) r n / (Ns R)}   (w_n = exp(-2 pi i / n); conj for inverse)
//   DFT_R in registers
//   outputs  y[(j - j mod Ns) R + j mod Ns + r Ns]
// and the last stage leaves the transform in natural order (self-sorting).  Stages run
// out of place between the tile and a scratch buffer ("ping-pong"); the butterflies of a
// stage are spread over all threads of the block and nothing is held in registers across a
// barrier.  The last stage writes exactly the positions it reads (j + r n/R), so it can put
// its result back into the tile from either buffer.
//
// Two tile layouts:
//   columns  element i of column col of component c at base[c * cs + i * NCOL + col]  (y and
//            z passes; a butterfly takes a pair of adjacent columns, consecutive threads take
//            consecutive pairs)
//   rows     element i of row `row` of component c at base[c * cs + row * ld + i]  (x passes;
//            consecutive threads take consecutive butterflies of a row)
// Divisions by the per-stage counts use float reciprocals (exact for the small integers here).
#pragma once
#include "cbs_internal.h"
#include "fft_radix.cuh"

#include <type_traits>

namespace cbs {

// Stage q of a plan: {r, Ns, stride = n/r, twstep = n/(Ns r)} and {1/stride, 1/Ns}.
__device__ __forceinline__ int4 stage_of(const AxisPlan& ap, int q) { return __ldg(&ap.st[2 * q]); }
__device__ __forceinline__ float2 stage_inv(const AxisPlan& ap, int q) {
  const int4 v = __ldg(&ap.st[2 * q + 1]);
  return make_float2(__int_as_float(v.x), __int_as_float(v.y));
}

// floor(k / d) for 0 <= k < 2^20 and 1 <= d <= 2^12 given inv = 1/d rounded to float:
// (k + 1/2)/d is at least 1/(2d) away from an integer, far more than the float rounding of
// the product.
__device__ __forceinline__ int fdiv(int k, float inv) { return __float2int_rz(((float)k + 0.5f) * inv); }

// tw: the axis' table w_n^m, m < n, in shared memory (copied in with the tile).  TW is false
// for a transform's first stage (Ns = 1: every twiddle is 1) and true for the others, where
// the butterflies with kk = 0 multiply by w^0 = (1, 0) exactly -- one branch per stage
// instead of a divergent one per butterfly.
template <int R, bool INV, bool TW>
__device__ __forceinline__ void twiddle_dft(float2* v, int kk, int twstep, const float2* tw) {
  if constexpr (R > 1 && TW) {
    const int step = kk * twstep;
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 w = tw[r * step];
      if (INV) w.y = -w.y;
      v[r] = cmul(v[r], w);
    }
  }
  DFT<R, INV>::run(v);
}

struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// ------------------------------------------------------------- column tiles, paired, multi-component
// Element (c, i, col) at base[c * cs + i * NCOL + col] (c < NCOMP).  An item transforms
// columns 2p and 2p+1 of one component together: 16-byte shared-memory accesses, one twiddle
// load and one set of index computations for both.  Items run p fastest, then j, then c.
template <int R, bool INV, int NCOL, int NCOMP, bool TW>
__device__ __forceinline__ void stage_cols2(const float2* src, float2* dst, int cs, int4 g, float2 iv,
                                            const float2* tw, int tid, int nth) {
  constexpr int NP = NCOL / 2;
  const int stride = g.z, Ns = g.y;
  const int items = NCOMP * NP * stride;
  for (int k = tid; k < items; k += nth) {
    const int p = (int)((unsigned)k % NP), rest = (int)((unsigned)k / NP);
    int c = 0, j = rest;
    if constexpr (NCOMP > 1) {
      c = fdiv(rest, iv.x);
      j = rest - c * stride;
    }
    const float4* s4 = reinterpret_cast<const float4*>(src + c * cs) + p;
    float2 v0[R], v1[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4 q = s4[(j + r * stride) * NP];
      v0[r] = make_float2(q.x, q.y);
      v1[r] = make_float2(q.z, q.w);
    }
    int qq = 0, kk = 0;
    if constexpr (TW) {
      qq = fdiv(j, iv.y);
      kk = j - qq * Ns;
    } else {
      qq = j;   // Ns = 1
    }
    if constexpr (R > 1 && TW) {
      const int step = kk * g.w;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = tw[r * step];
        if (INV) w.y = -w.y;
        v0[r] = cmul(v0[r], w);
        v1[r] = cmul(v1[r], w);
      }
    }
    DFT<R, INV>::run(v0);
    DFT<R, INV>::run(v1);
    const int d = qq * Ns * R + kk;
    float4* d4 = reinterpret_cast<float4*>(dst + c * cs) + p;
#pragma unroll
    for (int r = 0; r < R; ++r) d4[(d + r * Ns) * NP] = make_float4(v0[r].x, v0[r].y, v1[r].x, v1[r].y);
  }
}

// Stages [q0, q1) of the transform of NCOMP x NCOL columns whose stage-q0 input is in `in`
// (A or B; component stride cs), ping-ponging between A and B; a stage that is the last of
// the transform writes A (its outputs sit where it read them, so that is safe from either
// buffer).  Returns the buffer holding the output of stage q1 - 1.  Barrier after each stage;
// `after_first` runs after the first of them.
template <bool INV, int NCOL, int NCOMP, int MAXR = 16, class Hook = NoHook>
__device__ __forceinline__ float2* cols2_stages(float2* in, float2* A, float2* B, int cs, const AxisPlan& ap,
                                                int q0, int q1, const float2* tw, int tid, int nth,
                                                Hook after_first = Hook{}) {
  float2* src = in;
  for (int q = q0; q < q1; ++q) {
    const int4 g = stage_of(ap, q);
    const float2 iv = stage_inv(ap, q);
    float2* out = (q == ap.ns - 1) ? A : (src == A ? B : A);
    radix_dispatch<MAXR>(g.x, [&](auto Ri) {
      constexpr int R = decltype(Ri)::value;
      if (q == 0)
        stage_cols2<R, INV, NCOL, NCOMP, false>(src, out, cs, g, iv, tw, tid, nth);
      else
        stage_cols2<R, INV, NCOL, NCOMP, true>(src, out, cs, g, iv, tw, tid, nth);
    });
    __syncthreads();
    if (q == q0) after_first();
    src = out;
  }
  return src;
}

// ------------------------------------------------------------------- row tiles (x)
// Intermediate results of a row tile are stored swizzled: element A sits at
// A ^ ((A >> 4) & 15), which keeps every group of 16 in place (rows start on multiples of 16)
// and spreads the stride-R accesses of the early stages (Ns < 16) over all banks.
__device__ __forceinline__ int swz(int a) { return a ^ ((a >> 4) & 15); }

// Element hooks of a row transform.  Pre(c, row, x, v) gives the value the first stage uses
// for input element (c, row, x) (the forward x pass forms V E + S there, as it loads);
// Post(c, row, x, v) takes output element (c, row, x) of the last stage instead of a store
// (the inverse x pass updates E there).  NoPre / NoPost: plain loads and stores.
struct NoPre {
  __device__ __forceinline__ float2 operator()(int, int, int, float2 v) const { return v; }
};
struct NoPost {
  __device__ __forceinline__ void operator()(int, int, int, float2) const {}
};
// A Pre hook that makes its value from (c, row, x) alone: the first stage does not load its
// input from the tile (the fused x pass forms V E + S from another buffer).
template <class F>
struct Generate {
  F f;
  static constexpr bool kGenerates = true;
  __device__ __forceinline__ float2 operator()(int c, int row, int x, float2) const { return f(c, row, x); }
};
template <class F>
__device__ __forceinline__ Generate<F> generate(F f) { return Generate<F>{f}; }
template <class P, class = void>
struct generates : std::false_type {};
template <class P>
struct generates<P, std::void_t<decltype(P::kGenerates)>> : std::bool_constant<P::kGenerates> {};

template <int R, bool INV, bool TW, class Pre, class Post>
__device__ __forceinline__ void stage_rows(const float2* src, float2* dst, bool sw_in, bool sw_out, int nrows,
                                           int ncomp, int ld, int cs, int4 g, float2 iv,
                                           const float2* tw, int tid, int nth, Pre pre, Post post) {
  constexpr bool kPre = !std::is_same<Pre, NoPre>::value;
  constexpr bool kGen = generates<Pre>::value;
  constexpr bool kPost = !std::is_same<Post, NoPost>::value;
  const int stride = g.z, Ns = g.y;
  const int items = ncomp * nrows * stride;
  const float inv_rows = 1.0f / (float)nrows;
  for (int k = tid; k < items; k += nth) {
    const int t = fdiv(k, iv.x);           // (component, row) index
    const int j = k - t * stride;
    const int c = fdiv(t, inv_rows), row = t - c * nrows;
    const int base = c * cs + row * ld;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if constexpr (kGen) {
        v[r] = pre(c, row, j + r * stride, make_float2(0.f, 0.f));
      } else {
        const int a = base + j + r * stride;
        v[r] = src[sw_in ? swz(a) : a];
        if constexpr (kPre) v[r] = pre(c, row, j + r * stride, v[r]);
      }
    }
    int q = j, kk = 0;   // Ns = 1 in a first stage
    if constexpr (TW) {
      q = fdiv(j, iv.y);
      kk = j - q * Ns;
    }
    twiddle_dft<R, INV, TW>(v, kk, g.w, tw);
    const int d = q * Ns * R + kk;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if constexpr (kPost) {
        post(c, row, d + r * Ns, v[r]);
      } else {
        const int a = base + d + r * Ns;
        dst[sw_out ? swz(a) : a] = v[r];
      }
    }
  }
}

// FFT of nrows rows of ncomp components held in A (component stride cs, row stride ld; cs,
// ld and the base of A multiples of 16), scratch B of the same layout, with the element hooks
// pre (first stage) and post (last stage).  Returns the buffer holding the (unswizzled)
// result: A, or B when the last of several stages reads A (its swizzled reads and
// unswizzled writes must not share a buffer); nothing is stored when post is not NoPost.
// `after_first` runs in every thread after the first stage's barrier.  Ends with a barrier.
template <bool INV, int MAXR = 16, class Pre = NoPre, class Post = NoPost, class Hook = NoHook>
__device__ __forceinline__ float2* fft_rows(float2* A, float2* B, int nrows, int ncomp, int ld, int cs,
                                            const AxisPlan& ap, const float2* tw, int tid, int nth,
                                            Pre pre = Pre{}, Post post = Post{}, Hook after_first = Hook{}) {
  const int ns = ap.ns;
  float2* src = A;
  float2* dst = B;
  float2* out = A;
  for (int q = 0; q < ns; ++q) {
    const int4 g = stage_of(ap, q);
    const float2 iv = stage_inv(ap, q);
    const bool last = (q == ns - 1);
    out = !last ? dst : (q > 0 ? dst : A);
    radix_dispatch<MAXR>(g.x, [&](auto Ri) {
      constexpr int R = decltype(Ri)::value;
      if (q == 0 && last)
        stage_rows<R, INV, false>(src, out, false, false, nrows, ncomp, ld, cs, g, iv, tw, tid, nth, pre, post);
      else if (q == 0)
        stage_rows<R, INV, false>(src, out, false, true, nrows, ncomp, ld, cs, g, iv, tw, tid, nth, pre, NoPost{});
      else if (last)
        stage_rows<R, INV, true>(src, out, true, false, nrows, ncomp, ld, cs, g, iv, tw, tid, nth, NoPre{}, post);
      else
        stage_rows<R, INV, true>(src, out, true, true, nrows, ncomp, ld, cs, g, iv, tw, tid, nth, NoPre{}, NoPost{});
    });
    __syncthreads();
    if (q == 0) after_first();
    float2* t = src;
    src = dst;
    dst = t;
  }
  return out;
}

}  // namespace cbs
