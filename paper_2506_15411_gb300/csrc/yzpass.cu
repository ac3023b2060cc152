// yzpass.cu -- the strided passes of one CBS iteration.
//
//   y pass:  W_c <- FFT_y(W_c) or IFFT_y(W_c), one component per block
//   z pass:  W <- IFFT_z( G(p) FFT_z(W) ), the three components together, where
//            G(p) = (I - p p^T / kt2) / (|p|^2 - kt2), kt2 = k0^2 + i epsilon,
//            is the dyadic Green's function of curl curl - kt2 (the vector CBS of
//            refs. [25], [26] of arXiv 2506.15411), scaled by 1/N for the inverse FFT
//            (with the Nyquist treatment described at `Green`).
// A block owns TX consecutive x columns of one (z, c) plane (y pass) or of one y row (z
// pass); threads with consecutive x sit next to each other, so loads and stores move
// TX * 8 contiguous bytes per row.  The z pass transforms the three components of a column
// into shared memory, applies G(p) there (it mixes the components) and transforms back.
#include "stockham.cuh"

namespace cbs {

namespace {

__device__ __forceinline__ int fft_freq(int k, int n) { return (2 * k < n) ? k : k - n; }

template <bool INV>
__global__ void __launch_bounds__(512, 1) k_ypass(const IterArgs a) {
  extern __shared__ float2 smem[];
  const int TX = a.tx_y;
  const int tx = threadIdx.x % TX, t = threadIdx.x / TX;
  const int x = blockIdx.x * TX + tx;
  const int z = blockIdx.y, c = blockIdx.z;
  const bool ok = x < a.nx;
  const size_t nx = a.nx;
  float2* __restrict__ col = a.W + c * a.N + (size_t)z * a.ny * nx + (ok ? x : 0);
  SCol s{smem + tx, TX, 0};
  auto ld = [&](int, int i) -> float2 { return col[i * nx]; };
  auto st = [&](int, int i, float2 v) { col[i * nx] = v; };
  fft_columns<INV>(a.ay, 1, ld, st, s, t, ok, a.twy);
}

// k-space multiply at (kx, ky, kz):
//   X <- [X + q (q.X) / (|p|^2 - |q|^2 - kt2)] * invN / (|p|^2 - kt2),
// the inverse of |p|^2 I - q q^T - kt2 I, where q = p except that a Nyquist component (even
// axis length, wave number pi/pitch whose sign is undefined) is 0 in q, which keeps the
// discrete curl curl real and symmetric.  Away from Nyquist q = p and this is
// (I - p p^T / kt2) / (|p|^2 - kt2).
struct Green {
  float px, py, qx, qy, two_pi_nz;
  int nz;
  float2 kt2;
  float invN;
  __device__ __forceinline__ void operator()(int kz, float2& X0, float2& X1, float2& X2) const {
    const int fz = fft_freq(kz, nz);
    const float pz = two_pi_nz * (float)fz;
    const float qz = (2 * kz == nz) ? 0.f : pz;
    const float p2 = px * px + py * py + pz * pz;
    const float nyq2 = (px * px - qx * qx) + (py * py - qy * qy) + (pz * pz - qz * qz);
    // c = (q.X) / (nyq2 - kt2)
    const float cr = nyq2 - kt2.x, ci = -kt2.y;
    const float cs = 1.f / (cr * cr + ci * ci);
    const float2 qd = make_float2(qx * X0.x + qy * X1.x + qz * X2.x, qx * X0.y + qy * X1.y + qz * X2.y);
    const float2 c = cmul(qd, make_float2(cr * cs, -ci * cs));
    const float dr = p2 - kt2.x, di = -kt2.y;
    const float sc = invN / (dr * dr + di * di);
    const float2 inv = make_float2(dr * sc, -di * sc);   // invN / (dr + i di)
    X0 = cmul(make_float2(X0.x + qx * c.x, X0.y + qx * c.y), inv);
    X1 = cmul(make_float2(X1.x + qy * c.x, X1.y + qy * c.y), inv);
    X2 = cmul(make_float2(X2.x + qz * c.x, X2.y + qz * c.y), inv);
  }
};

__global__ void __launch_bounds__(512, 1) k_zpass_green(const IterArgs a) {
  extern __shared__ float2 smem[];
  const int TX = a.tx_z;
  const int tx = threadIdx.x % TX, t = threadIdx.x / TX;
  const int x = blockIdx.x * TX + tx;
  const int y = blockIdx.y;
  const bool ok = x < a.nx;
  const size_t plane = (size_t)a.nx * a.ny;
  const size_t N = a.N;
  float2* __restrict__ col = a.W + (size_t)y * a.nx + (ok ? x : 0);
  const int n = a.nz;
  SCol s{smem + tx, TX, n * TX};
  auto ld = [&](int c, int i) -> float2 { return col[c * N + i * plane]; };
  auto st = [&](int c, int i, float2 v) { col[c * N + i * plane] = v; };
  const float two_pi = 6.283185307179586f;
  Green gr;
  gr.px = two_pi / (float)a.nx * (float)fft_freq(x, a.nx);
  gr.py = two_pi / (float)a.ny * (float)fft_freq(y, a.ny);
  gr.qx = (2 * x == a.nx) ? 0.f : gr.px;
  gr.qy = (2 * y == a.ny) ? 0.f : gr.py;
  gr.two_pi_nz = two_pi / (float)n;
  gr.nz = n;
  gr.kt2 = a.kt2;
  gr.invN = a.invN;

  const AxisPlan& ap = a.az;
  const float2* __restrict__ tw = a.twz;
  const int ns = ap.ns;
  // forward FFT_z of the three components, left in natural order in shared memory
  {
    const int4 g = stage_of(ap, 0);
    radix_dispatch(g.x, [&](auto Ri) {
      constexpr int R = decltype(Ri)::value;
      stage_first_g<R, false>(ld, s, 0, 3, g.z, t, ok && t < g.z);
    });
  }
  __syncthreads();
  const int ql = ns - 1;
  for (int c = 0; c < 3 && ns > 1; ++c) {
    for (int q = 1; q < ql; ++q) {
      const int4 g = stage_of(ap, q);
      stage_mid<false>(g.x, s, c, g.z, g.y, g.w, t, ok && t < g.z, tw);
    }
    const int4 g = stage_of(ap, ql);
    radix_dispatch(g.x, [&](auto Ri) {
      constexpr int R = decltype(Ri)::value;
      stage_last_s<R, false>(s, c, g.z, g.y, g.w, t, ok && t < g.z, tw);
    });
  }
  __syncthreads();
  // k-space multiply, three components of one kz per step
  if (ok) {
    for (int i = t; i < n; i += ap.T) {
      float2 X0 = s.at(0, i), X1 = s.at(1, i), X2 = s.at(2, i);
      gr(i, X0, X1, X2);
      s.at(0, i) = X0;
      s.at(1, i) = X1;
      s.at(2, i) = X2;
    }
  }
  __syncthreads();
  // inverse FFT_z from shared memory (natural order) back to global memory
  for (int c = 0; c < 3; ++c) {
    for (int q = 0; q < ql; ++q) {
      const int4 g = stage_of(ap, q);
      stage_mid<true>(g.x, s, c, g.z, g.y, g.w, t, ok && t < g.z, tw);
    }
  }
  const int4 g = stage_of(ap, ql);
  radix_dispatch(g.x, [&](auto Ri) {
    constexpr int R = decltype(Ri)::value;
    stage_last_g<R, true>(st, s, 0, 3, g.z, g.y, g.w, t, ok && t < g.z, tw);
  });
}

}  // namespace

size_t ypass_smem(const IterArgs& a) { return (size_t)a.ny * a.tx_y * sizeof(float2); }
size_t zpass_smem(const IterArgs& a) { return (size_t)3 * a.nz * a.tx_z * sizeof(float2); }

cudaError_t launch_ypass(const IterArgs& a, bool inverse, cudaStream_t s) {
  dim3 grid((a.nx + a.tx_y - 1) / a.tx_y, a.nz, 3);
  const int threads = a.tx_y * a.ay.T;
  if (inverse)
    k_ypass<true><<<grid, threads, ypass_smem(a), s>>>(a);
  else
    k_ypass<false><<<grid, threads, ypass_smem(a), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_zpass_green(const IterArgs& a, cudaStream_t s) {
  dim3 grid((a.nx + a.tx_z - 1) / a.tx_z, a.ny, 1);
  k_zpass_green<<<grid, a.tx_z * a.az.T, zpass_smem(a), s>>>(a);
  return cudaGetLastError();
}

cudaError_t yzpass_set_smem_limit(int bytes) {
  cudaError_t e;
  e = cudaFuncSetAttribute(k_ypass<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_ypass<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_zpass_green, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace cbs
