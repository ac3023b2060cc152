// fft_host.cu -- runs the FFT stage code of the CUDA library (fft_ip.cuh, axis_plan.h) on the
// CPU, one emulated thread at a time, for the tests: a stage has no dependence between its
// items, so running thread 0, 1, ..., nth-1 in turn between the stages' barriers gives what
// the block computes.  Built for the host only (no device code); not part of the library.
#include <cstring>
#include <vector>

#include "axis_plan.h"
#include "fft_ip.cuh"

using namespace cbs;

namespace {

struct Axis {
  std::vector<int> order;
  std::vector<int4> st;
  std::vector<float2> tw, pq;
  AxisIP ap;
};

bool make_axis(int n, int layout, int ncol, Axis& A) {
  std::vector<int> rad;
  if (!factor_radices(n, 16, rad)) return false;
  A.order = order_radices(rad, n, (AxisLayout)layout, ncol);
  axis_tables(n, A.order, A.st, A.tw, A.pq);
  A.ap.n = n;
  A.ap.ns = (int)A.order.size();
  A.ap.st = A.st.data();
  if (A.tw.empty()) A.tw.push_back(make_float2(1.f, 0.f));
  return true;
}

template <class F>
void each_thread(int nth, F f) {
  for (int t = 0; t < nth; ++t) f(t);
}

// One column stage (NCOMP components, NCOL columns) of radix s.R, on column pairs or, with
// g_pairs off, on single columns.
bool g_pairs = true;

template <bool INV, int NCOL, int NCOMP>
void col_stage(float2* buf, int cs, const IPStage& s, bool tw_on, const float2* tw, int nth) {
  radix_dispatch<16>(s.R, [&](auto Ri) {
    constexpr int R = decltype(Ri)::value;
    each_thread(nth, [&](int t) {
      if (g_pairs) {
        if (tw_on)
          ipc_stage<R, INV, NCOL, NCOMP, true>(buf, cs, s, tw, t, nth);
        else
          ipc_stage<R, INV, NCOL, NCOMP, false>(buf, cs, s, tw, t, nth);
      } else {
        if (tw_on)
          ipc_stage1<R, INV, NCOL, NCOMP, true>(buf, cs, s, tw, t, nth);
        else
          ipc_stage1<R, INV, NCOL, NCOMP, false>(buf, cs, s, tw, t, nth);
      }
    });
  });
}

template <int NCOL, int NCOMP>
void cols_dif(float2* buf, int cs, const Axis& A, int q0, int q1, int nth) {
  for (int q = q0; q < q1; ++q)
    col_stage<false, NCOL, NCOMP>(buf, cs, ip_decode_stage(A.ap, q), q < A.ap.ns - 1, A.tw.data(), nth);
}
template <int NCOL, int NCOMP>
void cols_dit(float2* buf, int cs, const Axis& A, int q1, int q0, int nth) {
  for (int q = q1 - 1; q >= q0; --q)
    col_stage<true, NCOL, NCOMP>(buf, cs, ip_decode_stage(A.ap, q), q < A.ap.ns - 1, A.tw.data(), nth);
}

template <class F>
bool with_ncol(int ncol, F f) {
  switch (ncol) {
    case 2: f(std::integral_constant<int, 2>{}); return true;
    case 4: f(std::integral_constant<int, 4>{}); return true;
    case 8: f(std::integral_constant<int, 8>{}); return true;
    case 16: f(std::integral_constant<int, 16>{}); return true;
    default: return false;
  }
}

void row_stage(bool inv, float2* buf, int cs, int ld, int nrows, int ncomp, const IPStage& s, bool tw_on,
               const float2* tw, int nth) {
  radix_dispatch<16>(s.R, [&](auto Ri) {
    constexpr int R = decltype(Ri)::value;
    each_thread(nth, [&](int t) {
      if (inv) {
        if (tw_on) ipr_stage<R, true, true>(buf, cs, ld, nrows, ncomp, s, tw, t, nth);
        else ipr_stage<R, true, false>(buf, cs, ld, nrows, ncomp, s, tw, t, nth);
      } else {
        if (tw_on) ipr_stage<R, false, true>(buf, cs, ld, nrows, ncomp, s, tw, t, nth);
        else ipr_stage<R, false, false>(buf, cs, ld, nrows, ncomp, s, tw, t, nth);
      }
    });
  });
}

}  // namespace

extern "C" {

// Radix order of an axis for a layout (0 rows, 1 cols, 2 z cols); returns the stage count.
int fh_order(int n, int layout, int ncol, int* order) {
  Axis A;
  if (!make_axis(n, layout, ncol, A)) return -1;
  for (size_t i = 0; i < A.order.size(); ++i) order[i] = A.order[i];
  return (int)A.order.size();
}

// The z axis' order as the library picks it (radices up to 11 where the axis allows, then
// the least modelled work for nth threads on ncol-column tiles).
int fh_order_z(int n, int ncol, int nth, int* order) {
  std::vector<int> rad;
  if (!factor_radices(n, 11, rad) && !factor_radices(n, 16, rad)) return -1;
  const std::vector<int> o = order_radices_z(rad, n, ncol, nth);
  for (size_t i = 0; i < o.size(); ++i) order[i] = o[i];
  return (int)o.size();
}

// The z work model of an order (s radices).
long long fh_z_balance(int n, const int* order, int s, int ncol, int nth) {
  return z_balance_cost(std::vector<int>(order, order + s), n, ncol, nth);
}

// Wave numbers (p, q) per position (float2 [n]).
int fh_pq(int n, int layout, int ncol, float* pq) {
  Axis A;
  if (!make_axis(n, layout, ncol, A)) return -1;
  std::memcpy(pq, A.pq.data(), n * sizeof(float2));
  return 0;
}

// Columns: data complex64 [ncomp][n][ncol]; spec <- DIF(data); back <- DIT(spec); the stages
// work on column pairs (pairs != 0) or single columns.
int fh_cols(int n, int layout, int ncol, int ncomp, int nth, int pairs, const float* in, float* spec, float* back) {
  g_pairs = pairs != 0;
  Axis A;
  if (!make_axis(n, layout, ncol, A) || (ncomp != 1 && ncomp != 3)) return -1;
  const int cs = n * ncol;
  std::vector<float2> buf(ncomp * cs);
  std::memcpy(buf.data(), in, buf.size() * sizeof(float2));
  bool ok = with_ncol(ncol, [&](auto C) {
    constexpr int NC = decltype(C)::value;
    if (ncomp == 1) cols_dif<NC, 1>(buf.data(), cs, A, 0, A.ap.ns, nth);
    else cols_dif<NC, 3>(buf.data(), cs, A, 0, A.ap.ns, nth);
    std::memcpy(spec, buf.data(), buf.size() * sizeof(float2));
    if (ncomp == 1) cols_dit<NC, 1>(buf.data(), cs, A, A.ap.ns, 0, nth);
    else cols_dit<NC, 3>(buf.data(), cs, A, A.ap.ns, 0, nth);
  });
  if (!ok) return -2;
  std::memcpy(back, buf.data(), buf.size() * sizeof(float2));
  return 0;
}

// z pass on 3 components [3][n][ncol]: DIF stages 0..s-2, the fused stage with the point
// function X_c <- X_c * g(pos) (g: complex64 [n] per position), DIT stages s-2..0.
int fh_zpass(int n, int ncol, int nth, const float* in, const float* g, float* out) {
  g_pairs = true;
  Axis A;
  if (!make_axis(n, (int)AxisLayout::ColsZ, ncol, A)) return -1;
  const int cs = n * ncol;
  std::vector<float2> buf(3 * cs);
  std::memcpy(buf.data(), in, buf.size() * sizeof(float2));
  const float2* G = reinterpret_cast<const float2*>(g);
  const int s = A.ap.ns;
  bool ok = with_ncol(ncol, [&](auto C) {
    constexpr int NC = decltype(C)::value;
    cols_dif<NC, 3>(buf.data(), cs, A, 0, s - 1, nth);
    const IPStage st = ip_decode_stage(A.ap, s - 1);
    radix_dispatch<16>(st.R, [&](auto Ri) {
      constexpr int R = decltype(Ri)::value;
      each_thread(nth, [&](int t) {
        ipz_fused<R, NC>(buf.data(), cs, st, t, nth, [&](int, int pos, float2& X0, float2& X1, float2& X2) {
          X0 = cmul(X0, G[pos]);
          X1 = cmul(X1, G[pos]);
          X2 = cmul(X2, G[pos]);
        });
      });
    });
    cols_dit<NC, 3>(buf.data(), cs, A, s - 1, 0, nth);
  });
  if (!ok) return -2;
  std::memcpy(out, buf.data(), buf.size() * sizeof(float2));
  return 0;
}

// Rows: data complex64 [ncomp][nrows][ld] (row length n <= ld); spec <- DIF; back <- DIT.
int fh_rows(int n, int nrows, int ncomp, int ld, int nth, const float* in, float* spec, float* back) {
  Axis A;
  if (!make_axis(n, (int)AxisLayout::Rows, 0, A)) return -1;
  const int cs = nrows * ld;
  std::vector<float2> buf(ncomp * cs);
  std::memcpy(buf.data(), in, buf.size() * sizeof(float2));
  for (int q = 0; q < A.ap.ns; ++q)
    row_stage(false, buf.data(), cs, ld, nrows, ncomp, ip_decode_stage(A.ap, q), q < A.ap.ns - 1, A.tw.data(), nth);
  std::memcpy(spec, buf.data(), buf.size() * sizeof(float2));
  for (int q = A.ap.ns - 1; q >= 0; --q)
    row_stage(true, buf.data(), cs, ld, nrows, ncomp, ip_decode_stage(A.ap, q), q < A.ap.ns - 1, A.tw.data(), nth);
  std::memcpy(back, buf.data(), buf.size() * sizeof(float2));
  return 0;
}

// x pass on a spectrum [ncomp][nrows][ld] in DIF order: DIT stages s-1..1, the fused stage
// with u = a[x] * w + b[c][row][x] (a: complex64 [n]; b: complex64 [ncomp][nrows][ld]), DIF
// stages 1..s-1.
int fh_xpass(int n, int nrows, int ncomp, int ld, int nth, const float* spec, const float* a, const float* b,
             float* out) {
  Axis A;
  if (!make_axis(n, (int)AxisLayout::Rows, 0, A)) return -1;
  const int cs = nrows * ld;
  std::vector<float2> buf(ncomp * cs);
  std::memcpy(buf.data(), spec, buf.size() * sizeof(float2));
  const float2* Av = reinterpret_cast<const float2*>(a);
  const float2* Bv = reinterpret_cast<const float2*>(b);
  const int s = A.ap.ns;
  for (int q = s - 1; q >= 1; --q)
    row_stage(true, buf.data(), cs, ld, nrows, ncomp, ip_decode_stage(A.ap, q), q < s - 1, A.tw.data(), nth);
  const IPStage st = ip_decode_stage(A.ap, 0);
  radix_dispatch<16>(st.R, [&](auto Ri) {
    constexpr int R = decltype(Ri)::value;
    auto f = [&](int c, int row, int x, float2 w) { return cadd(cmul(Av[x], w), Bv[c * cs + row * ld + x]); };
    each_thread(nth, [&](int t) {
      if (s > 1) ipx_fused<R, true>(buf.data(), cs, ld, nrows, ncomp, st, A.tw.data(), t, nth, f);
      else ipx_fused<R, false>(buf.data(), cs, ld, nrows, ncomp, st, A.tw.data(), t, nth, f);
    });
  });
  for (int q = 1; q < s; ++q)
    row_stage(false, buf.data(), cs, ld, nrows, ncomp, ip_decode_stage(A.ap, q), q < s - 1, A.tw.data(), nth);
  std::memcpy(out, buf.data(), buf.size() * sizeof(float2));
  return 0;
}

}  // extern "C"
