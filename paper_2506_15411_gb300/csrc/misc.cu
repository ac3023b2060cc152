// misc.cu -- set-up, adjoint-source and gradient kernels.
//
//   set-up:    k^2 = k_vac^2 (eps_r + i sigma(r)),  k0^2 = (min Re k^2 + max Re k^2)/2,
//              epsilon = max |k^2 - k0^2| (FP64 block reductions),  V = k^2 - k0^2 - i epsilon
//              (splitting of the scalar CBS, ref. [25] of arXiv 2506.15411)
//   adjoint:   point source conj(E(r0)) at r0 for the figure of merit |E(r0)|^2 (Fig. 2 caption)
//   gradient:  dL/d eps_r = 2 k_vac^2 Re[E_adj . E]  (one pass over both fields)
// All k^2 quantities are in units of 1/pitch^2 (kv2 = (k_vac pitch)^2).
#include <cfloat>
#include <cstdint>
#include "absorber.h"
#include "cbs_internal.h"
#include "tma.cuh"

namespace cbs {

namespace {

template <class T, class Op>
__device__ __forceinline__ T block_reduce(T v, Op op, T* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = op(v, __shfl_down_sync(0xffffffffu, v, off));
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < nw; ++w) v = op(v, sh[w]);
  __syncthreads();
  return v;   // valid in thread 0
}

__global__ void k_eps_minmax(const float* __restrict__ eps, size_t N, float* pmin, float* pmax,
                             int* pbad) {
  __shared__ float sh[32];
  __shared__ int shi[32];
  float lo = FLT_MAX, hi = -FLT_MAX;
  int bad = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const float e = eps[i];
    if (!isfinite(e)) bad = 1;
    lo = fminf(lo, e);
    hi = fmaxf(hi, e);
  }
  lo = block_reduce(lo, [](float p, float q) { return fminf(p, q); }, sh);
  hi = block_reduce(hi, [](float p, float q) { return fmaxf(p, q); }, sh);
  bad = block_reduce(bad, [](int p, int q) { return p | q; }, shi);
  if (threadIdx.x == 0) {
    pmin[blockIdx.x] = lo;
    pmax[blockIdx.x] = hi;
    pbad[blockIdx.x] = bad;
  }
}

__device__ __forceinline__ void voxel_xyz(size_t i, int nx, int ny, int& x, int& y, int& z) {
  const size_t row = i / (size_t)nx;
  x = (int)(i - row * nx);
  z = (int)(row / (size_t)ny);
  y = (int)(row - (size_t)z * ny);
}

__global__ void k_k2_maxdev(const float* __restrict__ eps, int nx, int ny, int nz,
                            const double* __restrict__ sx, const double* __restrict__ sy,
                            const double* __restrict__ sz, int corner_max, double kv2, double k0sq,
                            double* part) {
  __shared__ double sh[32];
  const size_t N = (size_t)nx * ny * nz;
  double m = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    int x, y, z;
    voxel_xyz(i, nx, ny, x, y, z);
    const double re = kv2 * (double)eps[i] - k0sq;
    const double im = kv2 * layer_combine(sx[x], sy[y], sz[z], corner_max);
    m = fmax(m, re * re + im * im);   // squared: one square root per block, not per voxel
  }
  m = block_reduce(m, [](double p, double q) { return fmax(p, q); }, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = sqrt(m);   // sqrt is monotonic: the same maximum
}

// V in the y-blocked layout of the iteration (row padding stays zero).
__global__ void k_build_v(const float* __restrict__ eps, int nx, int ny, int nz, int nxp, int yblk,
                          const double* __restrict__ sx, const double* __restrict__ sy,
                          const double* __restrict__ sz, int corner_max, double kv2, double k0sq,
                          double eshift, float2* __restrict__ V) {
  const size_t N = (size_t)nx * ny * nz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    int x, y, z;
    voxel_xyz(i, nx, ny, x, y, z);
    const double re = kv2 * (double)eps[i] - k0sq;
    const double im = kv2 * layer_combine(sx[x], sy[y], sz[z], corner_max) - eshift;
    V[wrow(y, z, nz, yblk) * nxp + x] = make_float2((float)re, (float)im);
  }
}

// One thread per element of the 3 N field values, consecutive threads along x.
__global__ void k_field_layout(const float2* __restrict__ src, float2* __restrict__ dst, int to_dense, int nx, int ny,
                               int nz, int nxp, int yblk) {
  const size_t N = (size_t)nx * ny * nz, Nw = (size_t)nxp * ny * nz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < 3 * N; i += (size_t)gridDim.x * blockDim.x) {
    const size_t c = i / N, r = i - c * N;
    int x, y, z;
    voxel_xyz(r, nx, ny, x, y, z);
    const size_t b = c * Nw + wrow(y, z, nz, yblk) * nxp + x;
    if (to_dense)
      dst[i] = src[b];
    else
      dst[b] = src[i];
  }
}

__global__ void k_adjoint_amp(const float2* __restrict__ E, size_t N, size_t idx, float scale,
                              float2* amp) {
  if (threadIdx.x < 3) {
    const float2 e = E[threadIdx.x * N + idx];
    amp[threadIdx.x] = make_float2(e.x * scale, -e.y * scale);
  }
}

// Two voxels per thread through 16-byte loads when N is even; scalar tail otherwise.
__global__ void k_gradient(const float2* __restrict__ E, const float2* __restrict__ Ea, size_t N,
                           float coef, float* __restrict__ g, int vec) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  if (vec) {
    const size_t M = N / 2;
    const float4* E4 = reinterpret_cast<const float4*>(E);
    const float4* A4 = reinterpret_cast<const float4*>(Ea);
    float2* g2 = reinterpret_cast<float2*>(g);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < M; i += stride) {
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4 e = __ldg(&E4[c * M + i]);
        const float4 a = __ldg(&A4[c * M + i]);
        s0 = fmaf(a.x, e.x, fmaf(-a.y, e.y, s0));
        s1 = fmaf(a.z, e.z, fmaf(-a.w, e.w, s1));
      }
      g2[i] = make_float2(coef * s0, coef * s1);
    }
  } else {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += stride) {
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float2 e = __ldg(&E[c * N + i]);
        const float2 a = __ldg(&Ea[c * N + i]);
        s = fmaf(a.x, e.x, fmaf(-a.y, e.y, s));
      }
      g[i] = coef * s;
    }
  }
}

__global__ void k_objective(const float2* __restrict__ E, size_t N, size_t idx, double* out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int c = 0; c < 3; ++c) {
      const float2 e = E[c * N + idx];
      s += (double)e.x * e.x + (double)e.y * e.y;
    }
    *out = s;
  }
}

}  // namespace

cudaError_t launch_eps_minmax(const float* eps, size_t N, float* pmin, float* pmax, int* pbad,
                              int blocks, cudaStream_t s) {
  k_eps_minmax<<<blocks, 256, 0, s>>>(eps, N, pmin, pmax, pbad);
  return cudaGetLastError();
}

cudaError_t launch_k2_maxdev(const float* eps, int nx, int ny, int nz, const double* sx,
                             const double* sy, const double* sz, int corner_max, double kv2, double k0sq,
                             double* part, int blocks, cudaStream_t s) {
  k_k2_maxdev<<<blocks, 256, 0, s>>>(eps, nx, ny, nz, sx, sy, sz, corner_max, kv2, k0sq, part);
  return cudaGetLastError();
}

cudaError_t launch_build_v(const float* eps, int nx, int ny, int nz, int nxp, int yblk, const double* sx,
                           const double* sy, const double* sz, int corner_max, double kv2, double k0sq,
                           double eshift, float2* V, cudaStream_t s) {
  k_build_v<<<152 * 8, 256, 0, s>>>(eps, nx, ny, nz, nxp, yblk, sx, sy, sz, corner_max, kv2, k0sq, eshift, V);
  return cudaGetLastError();
}

cudaError_t launch_field_layout(const float2* src, float2* dst, bool to_dense, int nx, int ny, int nz, int nxp,
                                int yblk, cudaStream_t s) {
  k_field_layout<<<152 * 8, 256, 0, s>>>(src, dst, to_dense ? 1 : 0, nx, ny, nz, nxp, yblk);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_amp(const float2* E, size_t N, int nx, int ny, int x, int y, int z,
                               float scale, float2* amp, cudaStream_t s) {
  const size_t idx = ((size_t)z * ny + y) * nx + x;
  k_adjoint_amp<<<1, 32, 0, s>>>(E, N, idx, scale, amp);
  return cudaGetLastError();
}

cudaError_t launch_gradient(const float2* E, const float2* Ea, size_t N, float coef, float* g,
                            cudaStream_t s) {
  const int vec = (N % 2 == 0) && ((reinterpret_cast<uintptr_t>(E) | reinterpret_cast<uintptr_t>(Ea)) % 16 == 0) &&
                  (reinterpret_cast<uintptr_t>(g) % 8 == 0);
  k_gradient<<<152 * 8, 256, 0, s>>>(E, Ea, N, coef, g, vec);
  return cudaGetLastError();
}

cudaError_t launch_objective(const float2* E, size_t N, int nx, int ny, int x, int y, int z,
                             double* out, cudaStream_t s) {
  const size_t idx = ((size_t)z * ny + y) * nx + x;
  k_objective<<<1, 32, 0, s>>>(E, N, idx, out);
  return cudaGetLastError();
}

// Self-test of the bounded waits: an mbarrier that nothing arrives at, waited on with the
// tile kernels' bounded wait (`limit` polls).  The wait must give up, the kernel record the
// timeout in *err and return -- the error path every tile kernel takes instead of hanging.
__global__ void k_wait_selftest(int* err, long long limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit)) atomicExch(err, kErrTmaTimeout);
}

cudaError_t launch_wait_selftest(int* err, long long limit, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(err, limit);
  return cudaGetLastError();
}

}  // namespace cbs
