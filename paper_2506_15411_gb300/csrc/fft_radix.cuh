// fft_radix.cuh -- small in-register DFTs ("codelets") for the mixed-radix FFT passes.
//
// The 3D FFTs of the CBS iteration (the "N log N" cost of Fig. 1(b) of arXiv 2506.15411)
// are built from in-place DIF / DIT stages (fft_ip.cuh) whose butterflies are the DFTs below, applied to R values
// held in registers.  Supported radices: 1 (identity), 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12,
// 13, 16.
//   - odd primes: symmetric-pair form, X[k] and X[R-k] share the sums over the pairs
//     x[m] +- x[R-m] with real cos/sin constants;
//   - composites: one Cooley-Tukey split R = R1 * R2 (decimation in time) with the inner
//     twiddles as compile-time constants; quarter and eighth turns become swaps/negations.
// Constants come from a constexpr Taylor series in double precision, rounded to float.
#pragma once
#include <cuda_runtime.h>
#include <utility>

// The codelets also compile for the host (the tests run the FFT stages on the CPU).
#ifndef CBS_HD
#if defined(__CUDACC__)
#define CBS_HD __host__ __device__ __forceinline__
#else
#define CBS_HD inline
#endif
#endif

namespace cbs {

// ---------------------------------------------------------------- complex helpers
// The device code adds complex values with the packed FP32x2 instructions of sm_100+ (one
// instruction for both parts; the same IEEE results as two scalar adds; CBS_SCALAR_ADD turns
// them off).
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000 && !defined(CBS_SCALAR_ADD)
#define CBS_USE_PACKED 1
#else
#define CBS_USE_PACKED 0
#endif
CBS_HD float2 cadd(float2 a, float2 b) {
#if CBS_USE_PACKED
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
CBS_HD float2 csub(float2 a, float2 b) {
#if CBS_USE_PACKED
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}
// a + c b for real c, both parts
CBS_HD float2 cfma_r(float c, float2 b, float2 a) {
#if CBS_USE_PACKED
  return __ffma2_rn(make_float2(c, c), b, a);
#else
  return make_float2(fmaf(c, b.x, a.x), fmaf(c, b.y, a.y));
#endif
}
CBS_HD float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
CBS_HD float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
CBS_HD float2 mul_i(float2 a) { return make_float2(-a.y, a.x); }      //  i a
CBS_HD float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }     // -i a

// ---------------------------------------------------------------- compile-time loops
template <class F, int... I>
CBS_HD void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
CBS_HD void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ---------------------------------------------------------------- constexpr trigonometry
// cos and sin of 2 pi m / R from their Taylor series on [-pi, pi] (30 terms: the
// truncation error is far below double rounding there).
constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double ct_angle(int m, int R) {
  int mm = ((m % R) + R) % R;
  double a = 2.0 * kPi * (double)mm / (double)R;
  return a > kPi ? a - 2.0 * kPi : a;
}
constexpr double ct_sin(double x) {
  double term = x, sum = x;
  for (int n = 1; n < 30; ++n) {
    term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    sum += term;
  }
  return sum;
}
constexpr double ct_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 30; ++n) {
    term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}

// a * w_R^M with w_R = exp(-2 pi i / R) (forward) or exp(+2 pi i / R) (inverse).
template <int M, int R, bool INV>
CBS_HD float2 twc(float2 a) {
  constexpr int m = ((M % R) + R) % R;
  if constexpr (m == 0) {
    return a;
  } else if constexpr (2 * m == R) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (4 * m == R) {
    return INV ? mul_i(a) : mul_mi(a);
  } else if constexpr (4 * m == 3 * R) {
    return INV ? mul_mi(a) : mul_i(a);
  } else {
    constexpr float c = (float)ct_cos(ct_angle(m, R));
    constexpr float s = (float)(INV ? ct_sin(ct_angle(m, R)) : -ct_sin(ct_angle(m, R)));
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
  }
}

// ---------------------------------------------------------------- DFT codelets
template <int R, bool INV>
struct DFT;

template <bool INV>
struct DFT<1, INV> {
  static CBS_HD void run(float2*) {}
};

template <bool INV>
struct DFT<2, INV> {
  static CBS_HD void run(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

// Odd prime R: X[k] = A_k - i B_k, X[R-k] = A_k + i B_k (forward), with
// A_k = x0 + sum_m cos(2 pi k m / R)(x_m + x_{R-m}), B_k = sum_m sin(2 pi k m / R)(x_m - x_{R-m}).
template <int R, bool INV>
struct DFTOdd {
  static CBS_HD void run(float2* v) {
    constexpr int H = (R - 1) / 2;
    float2 a[H], b[H];
    float2 x0 = v[0];
    float2 sum = x0;
    static_for<H>([&](auto mi) {
      constexpr int m = decltype(mi)::value + 1;
      a[m - 1] = cadd(v[m], v[R - m]);
      b[m - 1] = csub(v[m], v[R - m]);
      sum = cadd(sum, a[m - 1]);
    });
    static_for<H>([&](auto ki) {
      constexpr int k = decltype(ki)::value + 1;
      float2 A = x0;
      float2 B = make_float2(0.f, 0.f);
      static_for<H>([&](auto mi) {
        constexpr int m = decltype(mi)::value + 1;
        constexpr float c = (float)ct_cos(ct_angle(k * m, R));
        constexpr float s = (float)ct_sin(ct_angle(k * m, R));
        A = cfma_r(c, a[m - 1], A);
        B = cfma_r(s, b[m - 1], B);
      });
      // forward: X[k] = A - iB = (A.x + B.y, A.y - B.x); X[R-k] = A + iB
      if constexpr (!INV) {
        v[k] = make_float2(A.x + B.y, A.y - B.x);
        v[R - k] = make_float2(A.x - B.y, A.y + B.x);
      } else {
        v[k] = make_float2(A.x - B.y, A.y + B.x);
        v[R - k] = make_float2(A.x + B.y, A.y - B.x);
      }
    });
    v[0] = sum;
  }
};

template <bool INV> struct DFT<3, INV> : DFTOdd<3, INV> {};
template <bool INV> struct DFT<5, INV> : DFTOdd<5, INV> {};
template <bool INV> struct DFT<7, INV> : DFTOdd<7, INV> {};
template <bool INV> struct DFT<11, INV> : DFTOdd<11, INV> {};
template <bool INV> struct DFT<13, INV> : DFTOdd<13, INV> {};

// Composite R = R1 * R2: input index n = R2 n1 + n2, output index k = k1 + R1 k2,
// X[k1 + R1 k2] = sum_n2 w_R2^{n2 k2} w_R^{n2 k1} sum_n1 x[R2 n1 + n2] w_R1^{n1 k1}.
template <int R1, int R2, bool INV>
struct DFTSplit {
  static constexpr int R = R1 * R2;
  static CBS_HD void run(float2* v) {
    float2 y[R];
    static_for<R2>([&](auto n2i) {
      constexpr int n2 = decltype(n2i)::value;
      float2 t[R1];
      static_for<R1>([&](auto n1i) {
        constexpr int n1 = decltype(n1i)::value;
        t[n1] = v[R2 * n1 + n2];
      });
      DFT<R1, INV>::run(t);
      static_for<R1>([&](auto k1i) {
        constexpr int k1 = decltype(k1i)::value;
        y[R2 * k1 + n2] = twc<n2 * k1, R, INV>(t[k1]);
      });
    });
    static_for<R1>([&](auto k1i) {
      constexpr int k1 = decltype(k1i)::value;
      float2 u[R2];
      static_for<R2>([&](auto n2i) {
        constexpr int n2 = decltype(n2i)::value;
        u[n2] = y[R2 * k1 + n2];
      });
      DFT<R2, INV>::run(u);
      static_for<R2>([&](auto k2i) {
        constexpr int k2 = decltype(k2i)::value;
        v[k1 + R1 * k2] = u[k2];
      });
    });
  }
};

template <bool INV> struct DFT<4, INV> : DFTSplit<2, 2, INV> {};
template <bool INV> struct DFT<6, INV> : DFTSplit<2, 3, INV> {};
template <bool INV> struct DFT<8, INV> : DFTSplit<2, 4, INV> {};
template <bool INV> struct DFT<9, INV> : DFTSplit<3, 3, INV> {};
template <bool INV> struct DFT<10, INV> : DFTSplit<2, 5, INV> {};
template <bool INV> struct DFT<12, INV> : DFTSplit<3, 4, INV> {};
template <bool INV> struct DFT<16, INV> : DFTSplit<4, 4, INV> {};

// Calls f(std::integral_constant<int, R>) for the runtime radix r (uniform across the block).
// Radices above MAXR are not compiled in (a plan whose axes need them uses a MAXR = 16
// kernel); leaving them out keeps the register allocation to what the smaller radices need.
template <int MAXR = 16, class F>
CBS_HD void radix_dispatch(int r, F&& f) {
  switch (r) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    case 7: f(std::integral_constant<int, 7>{}); break;
    case 8: f(std::integral_constant<int, 8>{}); break;
    case 9: if constexpr (MAXR >= 9) f(std::integral_constant<int, 9>{}); break;
    case 10: if constexpr (MAXR >= 10) f(std::integral_constant<int, 10>{}); break;
    case 11: if constexpr (MAXR >= 11) f(std::integral_constant<int, 11>{}); break;
    case 12: if constexpr (MAXR >= 12) f(std::integral_constant<int, 12>{}); break;
    case 13: if constexpr (MAXR >= 13) f(std::integral_constant<int, 13>{}); break;
    case 16: if constexpr (MAXR >= 16) f(std::integral_constant<int, 16>{}); break;
    default: break;
  }
}

}  // namespace cbs
