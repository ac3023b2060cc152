// xpass.cu -- the two passes along x (contiguous rows) of one CBS iteration.
//
//   forward:  W_c = FFT_x(V E_c + S_c)                       (scattering potential and source
//                                                              applied while loading)
//   inverse:  W_c = IFFT_x(W_c);  delta_c = gamma (E_c - W_c);  E_c -= delta_c;
//             sum |delta|^2 in FP64                           (update of the preconditioned
//                                                              series, refs. [25], [26] of
//                                                              arXiv 2506.15411)
// A block owns `rpb` rows (z, y) and all three components of each row (the three
// components of a voxel are handled by the same thread, so V is fetched from L1 after its
// first use).  T = nx / min(radix)
// threads per row; consecutive threads take consecutive x, so every global access is
// coalesced.
#include "stockham.cuh"

namespace cbs {

namespace {

__device__ __forceinline__ float2 source_at(const IterArgs& a, int c, int z, int y, int x, size_t idx) {
  const SourceArgs& s = a.src;
  if (s.kind == 0) {
    if (z == s.zp) return s.amp[c];
  } else if (s.kind == 1) {
    if (z == s.pz && y == s.py && x == s.px) return s.amp_dev ? s.amp_dev[c] : s.amp[c];
  } else {
    return cscale(__ldg(&s.user[c * a.N + idx]), s.user_scale);
  }
  return make_float2(0.f, 0.f);
}

// Block reduction of the per-thread residual in FP64, then a last-block-done pass that sums
// the per-block partials in a fixed order into hist[slot] (deterministic).
__device__ __forceinline__ void residual_finish(float acc, const IterArgs& a) {
  __shared__ double wsum[32];
  __shared__ bool last;
  double d = (double)acc;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  if (lane == 0) wsum[wid] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < nw; ++w) b += wsum[w];
    a.partials[blockIdx.x] = b;
    __threadfence();
    const unsigned prev = atomicAdd(a.counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(&a.partials[i]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  __syncthreads();
  if (lane == 0) wsum[wid] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < nw; ++w) b += wsum[w];
    a.hist[a.slot] = b;
    *a.counter = 0u;
  }
}

__global__ void __launch_bounds__(512, 1) k_xpass_fwd(const IterArgs a) {
  extern __shared__ float2 smem[];
  const int n = a.nx;
  const int T = a.ax.T;
  const int rl = threadIdx.x / T, t = threadIdx.x - rl * T;
  const int row = blockIdx.x * a.rpb + rl;
  const bool ok = row < a.ny * a.nz;
  const int z = row / a.ny, y = row - z * a.ny;
  const size_t base = (size_t)row * n;
  const float2* __restrict__ V = a.V;
  const float2* __restrict__ E = a.E;
  float2* __restrict__ W = a.W;
  const size_t N = a.N;
  SCol s{smem + (size_t)rl * 3 * n, 1, n};
  auto ld = [&](int c, int i) -> float2 {
    const size_t idx = base + i;
    return cadd(cmul(__ldg(&V[idx]), E[c * N + idx]), source_at(a, c, z, y, i, idx));
  };
  auto st = [&](int c, int i, float2 w) { W[c * N + base + i] = w; };
  fft_columns<false>(a.ax, 3, ld, st, s, t, ok, a.twx);
}

__global__ void __launch_bounds__(512, 1) k_xpass_inv_update(const IterArgs a) {
  extern __shared__ float2 smem[];
  const int n = a.nx;
  const int T = a.ax.T;
  const int rl = threadIdx.x / T, t = threadIdx.x - rl * T;
  const int row = blockIdx.x * a.rpb + rl;
  const bool ok = row < a.ny * a.nz;
  const size_t base = (size_t)row * n;
  const float2* __restrict__ V = a.V;
  float2* __restrict__ E = a.E;
  const float2* __restrict__ W = a.W;
  const size_t N = a.N;
  const float ie = a.inv_eps;
  float acc = 0.f;
  SCol s{smem + (size_t)rl * 3 * n, 1, n};
  auto ld = [&](int c, int i) -> float2 { return W[c * N + base + i]; };
  auto st = [&](int c, int i, float2 w) {
    const size_t idx = base + i;
    const float2 v = __ldg(&V[idx]);
    const float2 g = make_float2(-v.y * ie, v.x * ie);   // gamma = (i / epsilon) V
    const float2 e = E[c * N + idx];
    const float2 d = cmul(g, csub(e, w));
    E[c * N + idx] = csub(e, d);
    acc = fmaf(d.x, d.x, fmaf(d.y, d.y, acc));
  };
  fft_columns<true>(a.ax, 3, ld, st, s, t, ok, a.twx);
  residual_finish(acc, a);
}

}  // namespace

size_t xpass_smem(const IterArgs& a) { return (size_t)a.rpb * 3 * a.nx * sizeof(float2); }
int xpass_blocks(const IterArgs& a) { return (a.ny * a.nz + a.rpb - 1) / a.rpb; }

cudaError_t launch_xpass_fwd(const IterArgs& a, cudaStream_t s) {
  k_xpass_fwd<<<xpass_blocks(a), a.rpb * a.ax.T, xpass_smem(a), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_xpass_inv_update(const IterArgs& a, cudaStream_t s) {
  k_xpass_inv_update<<<xpass_blocks(a), a.rpb * a.ax.T, xpass_smem(a), s>>>(a);
  return cudaGetLastError();
}

cudaError_t xpass_set_smem_limit(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_xpass_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_xpass_inv_update, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace cbs
