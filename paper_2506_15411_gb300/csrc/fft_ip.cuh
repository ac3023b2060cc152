// fft_ip.cuh -- block-cooperative in-place mixed-radix FFT stages over tiles in shared memory.
//
// Forward transforms are decimation in frequency (DIF), inverse ones decimation in time (DIT),
// both in place.  For n = R_0 R_1 ... R_{s-1}, DIF stage q works on blocks of L_q = R_q m_q
// consecutive elements with m_q = n / (R_0 ... R_q); its butterfly (b, j), j < m_q, takes
// the R_q elements at b L_q + j + r m_q, applies DFT_R and multiplies output k by
// w_n^{j k P_q} (w_n = exp(-2 pi i / n), P_q = n / L_q), writing it back at b L_q + j + k m_q --
// the positions it read.  After the last stage, frequency k sits at the mixed-radix digit
// reversal of k:
//     k = d_0 + R_0 d_1 + R_0 R_1 d_2 + ...   ->   position sum_q d_q m_q.
// The DIT stages undo the DIF stages in reverse order (conjugate twiddles, then an inverse
// DFT_R), so DIT after DIF is n times the identity, and a pointwise multiply applied in
// between at position pos(k) with the value belonging to frequency k makes the pair a
// convolution: nothing is ever permuted.  The k-space multiply looks up the wave number of
// each position in a per-axis table the host builds.
//
// A butterfly reads and writes the same positions and no two butterflies of a stage share a
// position, so a stage needs no scratch buffer and no barrier inside it; the caller puts one
// barrier between stages.  The last DIF stage (m = 1) has no twiddles.
//
// Per-axis device tables, built by the host:
//   stages  two int4 per DIF stage q: {R, m, L, tw_off} and {bits of 1/m, bits of 1/(n/R), n/R, 0}
//           (float reciprocals for exact small-integer division);
//   tw      per stage q < s-1, the twiddles w_n^{j k P_q} at tw_off + (k - 1) m + j
//           (k = 1..R-1, j < m): consecutive butterflies read consecutive entries;
//   pq      per position, the wave number (p, q) of the frequency stored there (scaled by the
//           pitch; q = p except 0 at the Nyquist frequency of an even axis).
//
// Tile layouts, as in the passes:
//   columns  element i of column col of component c at base[c * cs + i * NCOL + col]  (y and
//            z passes; an item transforms a pair of adjacent columns with 16-byte accesses)
//   rows     element i of row `row` of component c at base[c * cs + row * ld + i]  (x passes;
//            consecutive items take consecutive butterflies of a row)
// Everything here is __host__ __device__ so that the host can run the same stage code one
// "thread" at a time to check it (the tests build it for the CPU).
#pragma once
#include <cuda_runtime.h>

#include <cstring>

#include "fft_radix.cuh"   // defines CBS_HD

namespace cbs {

// Device copy of one axis' plan.
struct AxisIP {
  int n;
  int ns;
  const int4* st;   // 2 * ns entries
};

CBS_HD float ip_bits_float(int b) {
#if defined(__CUDA_ARCH__)
  return __int_as_float(b);
#else
  float f;
  std::memcpy(&f, &b, sizeof(f));
  return f;
#endif
}

CBS_HD int4 ip_stage(const AxisIP& ap, int q) {
#if defined(__CUDA_ARCH__)
  return __ldg(&ap.st[2 * q]);
#else
  return ap.st[2 * q];
#endif
}
CBS_HD int4 ip_stage_aux(const AxisIP& ap, int q) {
#if defined(__CUDA_ARCH__)
  return __ldg(&ap.st[2 * q + 1]);
#else
  return ap.st[2 * q + 1];
#endif
}

// floor(k / d) for 0 <= k < 2^20, 1 <= d <= 2^12, inv = 1/d rounded to float: (k + 1/2)/d is
// at least 1/(2d) away from an integer, far more than the rounding of the product.
CBS_HD int ip_div(int k, float inv) {
#if defined(__CUDA_ARCH__)
  return __float2int_rz(((float)k + 0.5f) * inv);
#else
  return (int)(((float)k + 0.5f) * inv);
#endif
}

CBS_HD float2 ip_conj(float2 a) { return make_float2(a.x, -a.y); }

struct NoHookIP {
  CBS_HD void operator()() const {}
};

// Decoded item of a stage: butterfly t = b m + j of an axis.
struct IPStage {
  int R, m, L, twoff, nb;
  float inv_m, inv_nb;
};
CBS_HD IPStage ip_decode_stage(const AxisIP& ap, int q) {
  const int4 g = ip_stage(ap, q), a = ip_stage_aux(ap, q);
  IPStage s;
  s.R = g.x;
  s.m = g.y;
  s.L = g.z;
  s.twoff = g.w;
  s.inv_m = ip_bits_float(a.x);
  s.inv_nb = ip_bits_float(a.y);
  s.nb = a.z;
  return s;
}

// DIF butterfly: DFT_R, then output k times tw[(k-1) m + j] (the twiddles of this stage and
// butterfly; pass tw already offset by twoff + j, stride m).  TW = false: the last stage.
template <int R, bool TW>
CBS_HD void dif_bfly(float2* v, const float2* tw, int m) {
  DFT<R, false>::run(v);
  if constexpr (TW && R > 1) {
#pragma unroll
    for (int k = 1; k < R; ++k) v[k] = cmul(v[k], tw[(k - 1) * m]);
  }
}
// DIT butterfly: input k times conj(tw[(k-1) m + j]), then the inverse DFT_R.
template <int R, bool TW>
CBS_HD void dit_bfly(float2* v, const float2* tw, int m) {
  if constexpr (TW && R > 1) {
#pragma unroll
    for (int k = 1; k < R; ++k) v[k] = cmul(v[k], ip_conj(tw[(k - 1) * m]));
  }
  DFT<R, true>::run(v);
}

// --------------------------------------------------------------------- column tiles, paired
// One DIF (INV = false) or DIT (INV = true) stage over NCOMP x NCOL columns in `buf`
// (component stride cs).  Items run over (column pair p fastest, then butterfly t, then
// component c).
template <int R, bool INV, int NCOL, int NCOMP, bool TW>
CBS_HD void ipc_stage(float2* buf, int cs, const IPStage& s, const float2* tw, int tid, int nth) {
  constexpr int NP = NCOL / 2;
  const int m = s.m;
  const int items = NCOMP * NP * s.nb;
  for (int k = tid; k < items; k += nth) {
    const int p = (int)((unsigned)k % NP), rest = (int)((unsigned)k / NP);
    int c = 0, t = rest;
    if constexpr (NCOMP > 1) {
      c = ip_div(rest, s.inv_nb);
      t = rest - c * s.nb;
    }
    const int b = ip_div(t, s.inv_m), j = t - b * m;
    float4* q4 = reinterpret_cast<float4*>(buf + c * cs) + (b * s.L + j) * NP + p;
    const int rs = m * NP;
    float2 v0[R], v1[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4 q = q4[r * rs];
      v0[r] = make_float2(q.x, q.y);
      v1[r] = make_float2(q.z, q.w);
    }
    const float2* w = tw + s.twoff + j;
    if constexpr (!INV) {
      DFT<R, false>::run(v0);
      DFT<R, false>::run(v1);
      if constexpr (TW && R > 1) {
#pragma unroll
        for (int kk = 1; kk < R; ++kk) {
          const float2 ww = w[(kk - 1) * m];
          v0[kk] = cmul(v0[kk], ww);
          v1[kk] = cmul(v1[kk], ww);
        }
      }
    } else {
      if constexpr (TW && R > 1) {
#pragma unroll
        for (int kk = 1; kk < R; ++kk) {
          const float2 ww = ip_conj(w[(kk - 1) * m]);
          v0[kk] = cmul(v0[kk], ww);
          v1[kk] = cmul(v1[kk], ww);
        }
      }
      DFT<R, true>::run(v0);
      DFT<R, true>::run(v1);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) q4[r * rs] = make_float4(v0[r].x, v0[r].y, v1[r].x, v1[r].y);
  }
}

// The same stage on single columns (8-byte accesses, half the registers of the paired form):
// items run over (column fastest, then butterfly t, then component c).
template <int R, bool INV, int NCOL, int NCOMP, bool TW>
CBS_HD void ipc_stage1(float2* buf, int cs, const IPStage& s, const float2* tw, int tid, int nth) {
  const int m = s.m;
  const int items = NCOMP * NCOL * s.nb;
  for (int k = tid; k < items; k += nth) {
    const int col = (int)((unsigned)k % NCOL), rest = (int)((unsigned)k / NCOL);
    int c = 0, t = rest;
    if constexpr (NCOMP > 1) {
      c = ip_div(rest, s.inv_nb);
      t = rest - c * s.nb;
    }
    const int b = ip_div(t, s.inv_m), j = t - b * m;
    float2* q = buf + c * cs + (b * s.L + j) * NCOL + col;
    const int rs = m * NCOL;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = q[r * rs];
    if constexpr (!INV)
      dif_bfly<R, TW>(v, tw + s.twoff + j, m);
    else
      dit_bfly<R, TW>(v, tw + s.twoff + j, m);
#pragma unroll
    for (int r = 0; r < R; ++r) q[r * rs] = v[r];
  }
}

// --------------------------------------------------------------------------------- row tiles
// One DIF / DIT stage over ncomp x nrows rows in `buf` (component stride cs, row stride ld).
// Items run over (butterfly t fastest, then row, then component).  In the last DIF stage
// (m = 1) a butterfly's R elements are contiguous; for even R they move as float4 pairs.
template <int R, bool INV, bool TW>
CBS_HD void ipr_stage(float2* buf, int cs, int ld, int nrows, int ncomp, const IPStage& s, const float2* tw,
                      int tid, int nth) {
  const int m = s.m;
  const float inv_rows = 1.0f / (float)nrows;
  const int items = ncomp * nrows * s.nb;
  for (int k = tid; k < items; k += nth) {
    const int cr = ip_div(k, s.inv_nb);
    const int t = k - cr * s.nb;
    const int c = ip_div(cr, inv_rows), row = cr - c * nrows;
    const int b = ip_div(t, s.inv_m), j = t - b * m;
    float2* q = buf + c * cs + row * ld + b * s.L + j;
    float2 v[R];
    if constexpr (!TW && R % 2 == 0) {
      const float4* q4 = reinterpret_cast<const float4*>(q);
#pragma unroll
      for (int r = 0; r < R / 2; ++r) {
        const float4 u = q4[r];
        v[2 * r] = make_float2(u.x, u.y);
        v[2 * r + 1] = make_float2(u.z, u.w);
      }
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = q[r * m];
    }
    if constexpr (!INV)
      dif_bfly<R, TW>(v, tw + s.twoff + j, m);
    else
      dit_bfly<R, TW>(v, tw + s.twoff + j, m);
    if constexpr (!TW && R % 2 == 0) {
      float4* q4 = reinterpret_cast<float4*>(q);
#pragma unroll
      for (int r = 0; r < R / 2; ++r) q4[r] = make_float4(v[2 * r].x, v[2 * r].y, v[2 * r + 1].x, v[2 * r + 1].y);
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) q[r * m] = v[r];
    }
  }
}

// The first DIF stage of rows whose input is formed from (c, row, x) and the value held at
// that position (the forward x passes form V E + S there): gen(c, row, x, v) returns the
// value to transform.  In place; TW = false when the axis has one stage.
template <int R, bool TW, class G>
CBS_HD void ipr_dif_first(float2* buf, int cs, int ld, int nrows, int ncomp, const IPStage& s, const float2* tw,
                          int tid, int nth, G gen) {
  const int m = s.m;
  const float inv_rows = 1.0f / (float)nrows;
  const int items = ncomp * nrows * m;   // stage 0: L = n, one block of m butterflies per row
  for (int k = tid; k < items; k += nth) {
    const int cr = ip_div(k, s.inv_m);
    const int j = k - cr * m;
    const int c = ip_div(cr, inv_rows), row = cr - c * nrows;
    float2* q = buf + c * cs + row * ld + j;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = gen(c, row, j + r * m, q[r * m]);
    dif_bfly<R, TW>(v, tw + s.twoff + j, m);
#pragma unroll
    for (int r = 0; r < R; ++r) q[r * m] = v[r];
  }
}

// ------------------------------------------------------------------- fused middle stages
// z pass: the last DIF stage (m = 1, no twiddles), a point function on the three components
// at each of its R outputs, and the first DIT stage (its inverse) on the same R positions,
// all in registers.  Single columns of NCOL-column tiles of 3 components; items run over
// (column fastest, then butterfly b).  point(col, pos, X0, X1, X2) gets the transformed
// values at axis position pos (frequency by the axis' digit reversal) and updates them.
template <int R, int NCOL, class F>
CBS_HD void ipz_fused(float2* buf, int cs, const IPStage& s, int tid, int nth, F point) {
  const int items = NCOL * s.nb;
  for (int k = tid; k < items; k += nth) {
    const int col = (int)((unsigned)k % NCOL), b = (int)((unsigned)k / NCOL);
    float2* q = buf + b * R * NCOL + col;
    float2 v[3][R];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[c][r] = q[c * cs + r * NCOL];
      DFT<R, false>::run(v[c]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) point(col, b * R + r, v[0][r], v[1][r], v[2][r]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      DFT<R, true>::run(v[c]);
#pragma unroll
      for (int r = 0; r < R; ++r) q[c * cs + r * NCOL] = v[c][r];
    }
  }
}

// x pass: the last DIT stage (inverse of DIF stage 0: L = n, butterfly j < m = n/R), a
// function of each natural-order output, and DIF stage 0 on the function's values at the
// same positions, all in registers.  Rows of ncomp components; items run over (butterfly j
// fastest, then row, then component).  f(c, row, x, w) gets the inverse transform's value w
// at natural position x and returns the input of the forward transform there.  TW = false
// when stage 0 is the only stage (then it has no twiddles).
template <int R, bool TW, class F>
CBS_HD void ipx_fused(float2* buf, int cs, int ld, int nrows, int ncomp, const IPStage& s, const float2* tw,
                      int tid, int nth, F f) {
  const int m = s.m;
  const float inv_rows = 1.0f / (float)nrows;
  const int items = ncomp * nrows * m;
  for (int k = tid; k < items; k += nth) {
    const int cr = ip_div(k, s.inv_m);
    const int j = k - cr * m;
    const int c = ip_div(cr, inv_rows), row = cr - c * nrows;
    float2* q = buf + c * cs + row * ld + j;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = q[r * m];
    dit_bfly<R, TW>(v, tw + s.twoff + j, m);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = f(c, row, j + r * m, v[r]);
    dif_bfly<R, TW>(v, tw + s.twoff + j, m);
#pragma unroll
    for (int r = 0; r < R; ++r) q[r * m] = v[r];
  }
}

// Calls f(std::integral_constant<int, R>) for the runtime radix r (uniform across the block).
// Radices above MAXR are not compiled in (a plan whose axes need them uses a MAXR = 16
// kernel); leaving them out keeps the register allocation to what the smaller radices need.
template <int MAXR = 16, class F>
CBS_HD void ip_radix(int r, F&& f) {
  radix_dispatch<MAXR>(r, f);
}

}  // namespace cbs
