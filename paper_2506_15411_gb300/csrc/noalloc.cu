// noalloc.cu -- the splitting of a permittivity grid computed without allocating memory.
//
// cbs_splitting_noalloc (include/cbs.h) runs variants of the set-up reductions of
// misc.cu: the min/max of eps_r and max |k^2 - k0^2|, with k^2 = k_vac^2 (eps_r + i sigma)
// and the absorbing-layer profile sigma computed in the kernel from the pad widths.  Their
// per-block partial sums live in the file-scope device array g_scratch below instead of in
// plan-owned buffers, so the call needs no cudaMalloc: it serves callers that cannot
// allocate device memory, e.g. code whose device memory is handed out entirely by another
// allocator, or host loops that must not pay for (or synchronise on) cudaMalloc/cudaFree.
//
// g_scratch is one array per device that loads this library, held until the process exits;
// every call on a device shares it and leaves its contents behind.  Calls that overlap on
// the GPU (different streams or threads) race on it.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/cbs.h"
#include "absorber.h"

namespace cbs {
const char* set_last_error(const char* msg);   // api.cu
}

namespace {

constexpr int kMaxBlocks = 4096;                 // partial sums held in the scratch array
constexpr long long kVoxelsPerBlock = 65536;     // each block reduces one chunk of the grid
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;
constexpr int kMaxAxis = 1024;                   // longest axis cbs_plan accepts

struct Scratch {
  float pmin[kMaxBlocks];
  float pmax[kMaxBlocks];
  int pbad[kMaxBlocks];
  double pdev[kMaxBlocks];
  unsigned counter;       // last-block-done counter; cleared by the host before each kernel
  double lo, hi;          // min / max of eps_r
  int bad;                // any non-finite eps_r
  double k0sq, maxdev;    // scaled units (k^2 times pitch^2)
};

// About 80 KB on every device that loads the library.
static __device__ __align__(256) Scratch g_scratch;

struct LayerArgs {
  int n[3], lo[3], hi[3];
  double smax_lo[3], smax_hi[3];  // sigma_max of each face (0 where there is no layer)
  double power;                   // ramp exponent
  int corner_max;                 // overlapping layers: 0 add, 1 the largest
  double kv2;                     // (k_vac pitch)^2
};

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

// Returns true in the block that finished last (its partial writes are visible to it).
__device__ __forceinline__ bool last_block(Scratch* s) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&s->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

__global__ void k_noalloc_minmax(const float* __restrict__ eps, long long N, Scratch* s) {
  __shared__ float sh[32];
  __shared__ int shi[32];
  const long long b0 = blockIdx.x * kVoxelsPerBlock;
  const long long b1 = min(N, b0 + kVoxelsPerBlock);
  float lo = FLT_MAX, hi = -FLT_MAX;
  int bad = 0;
  for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const float e = eps[i];
    if (!isfinite(e)) bad = 1;
    lo = fminf(lo, e);
    hi = fmaxf(hi, e);
  }
  lo = block_reduce(lo, [](float p, float q) { return fminf(p, q); }, sh);
  hi = block_reduce(hi, [](float p, float q) { return fmaxf(p, q); }, sh);
  bad = block_reduce(bad, [](int p, int q) { return p | q; }, shi);
  if (threadIdx.x == 0) {
    s->pmin[blockIdx.x] = lo;
    s->pmax[blockIdx.x] = hi;
    s->pbad[blockIdx.x] = bad;
  }
  if (!last_block(s)) return;
  if (threadIdx.x == 0) {
    double mn = 1e300, mx = -1e300;
    int any = 0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
      mn = fmin(mn, (double)__ldcg(&s->pmin[b]));
      mx = fmax(mx, (double)__ldcg(&s->pmax[b]));
      any |= __ldcg(&s->pbad[b]);
    }
    s->lo = mn;
    s->hi = mx;
    s->bad = any;
  }
}

__global__ void k_noalloc_maxdev(const float* __restrict__ eps, long long N, LayerArgs L, Scratch* s) {
  __shared__ double sh[32];
  // k0^2 from the first kernel's extremes, the same expression as the plan's set-up
  const double k0sq = 0.5 * L.kv2 * (s->lo + s->hi);
  const long long b0 = blockIdx.x * kVoxelsPerBlock;
  const long long b1 = min(N, b0 + kVoxelsPerBlock);
  double m = 0.0;
  for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const long long row = i / L.n[0];
    const int x = (int)(i - row * L.n[0]);
    const int z = (int)(row / L.n[1]);
    const int y = (int)(row - (long long)z * L.n[1]);
    const double sx = cbs::layer_axis_sigma(x, L.n[0], L.lo[0], L.hi[0], L.smax_lo[0], L.smax_hi[0], L.power);
    const double sy = cbs::layer_axis_sigma(y, L.n[1], L.lo[1], L.hi[1], L.smax_lo[1], L.smax_hi[1], L.power);
    const double sz = cbs::layer_axis_sigma(z, L.n[2], L.lo[2], L.hi[2], L.smax_lo[2], L.smax_hi[2], L.power);
    const double re = L.kv2 * (double)eps[i] - k0sq;
    const double im = L.kv2 * cbs::layer_combine(sx, sy, sz, L.corner_max);
    m = fmax(m, sqrt(re * re + im * im));
  }
  m = block_reduce(m, [](double p, double q) { return fmax(p, q); }, sh);
  if (threadIdx.x == 0) s->pdev[blockIdx.x] = m;
  if (!last_block(s)) return;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) mx = fmax(mx, __ldcg(&s->pdev[b]));
    s->k0sq = k0sq;
    s->maxdev = mx;
  }
}

// Device address of g_scratch, looked up once per device with that device current (the
// primary context's copy of the array; a cudaDeviceReset ends that context, and the cached
// address with it -- the header says so).
std::mutex g_mu;
Scratch* g_ptr[kMaxDevices] = {};

cudaError_t scratch_for_device(int dev, Scratch** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = static_cast<Scratch*>(p);
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

int err(int code, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  cbs::set_last_error(buf);
  return code;
}

}  // namespace

extern "C" int cbs_splitting_noalloc(const cbs_plan_desc* d, const float* eps_real_dev, double* k0sq,
                                     double* epsilon) {
  cbs::set_last_error("");
  if (!d || !eps_real_dev || !k0sq || !epsilon) return err(CBS_ERR_ARG, "NULL argument");
  // the descriptor checks of cbs_plan, so that both entry points accept the same grids
  const int dims[3] = {d->nx, d->ny, d->nz};
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < 1 || dims[a] > kMaxAxis)
      return err(CBS_ERR_ARG, "axis %d size %d outside [1, %d]", a, dims[a], kMaxAxis);
    if (d->pad_lo[a] < 0 || d->pad_hi[a] < 0 || 2 * d->pad_lo[a] > dims[a] || 2 * d->pad_hi[a] > dims[a] ||
        d->pad_lo[a] + d->pad_hi[a] >= dims[a])
      return err(CBS_ERR_ARG, "axis %d pads (%d, %d) do not fit size %d", a, d->pad_lo[a], d->pad_hi[a], dims[a]);
  }
  if (!(d->pitch_m > 0) || !(d->lambda_m > 0) || !(d->n_bg > 0))
    return err(CBS_ERR_ARG, "pitch, wavelength and n_bg must be positive");
  const cbs::LayerSpec layers = cbs::layer_spec(d->layer_round_trip, d->layer_power, d->layer_corner_max);
  if (!cbs::layer_spec_valid(layers))
    return err(CBS_ERR_ARG, "layer round trip %g, power %g or corner rule %d out of range", d->layer_round_trip,
               d->layer_power, d->layer_corner_max);
  const long long N = (long long)d->nx * d->ny * d->nz;
  const long long blocks = (N + kVoxelsPerBlock - 1) / kVoxelsPerBlock;
  if (blocks > kMaxBlocks)
    return err(CBS_ERR_ARG, "grid of %lld voxels exceeds the no-alloc limit of %lld voxels", N,
               (long long)kMaxBlocks * kVoxelsPerBlock);

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  Scratch* s = nullptr;
  if (e == cudaSuccess) e = scratch_for_device(dev, &s);
  if (e != cudaSuccess) return err(CBS_ERR_CUDA, "scratch set-up failed: %s", cudaGetErrorString(e));

  const double kPi = 3.14159265358979323846;
  const double kvac = 2.0 * kPi / d->lambda_m;
  LayerArgs L{};
  for (int a = 0; a < 3; ++a) {
    L.n[a] = dims[a];
    L.lo[a] = d->pad_lo[a];
    L.hi[a] = d->pad_hi[a];
    L.smax_lo[a] = cbs::layer_sigma_max(layers, d->n_bg, kvac, d->pad_lo[a], d->pitch_m);
    L.smax_hi[a] = cbs::layer_sigma_max(layers, d->n_bg, kvac, d->pad_hi[a], d->pitch_m);
  }
  L.power = layers.power;
  L.corner_max = layers.corner_max;
  L.kv2 = (kvac * d->pitch_m) * (kvac * d->pitch_m);

  cudaStream_t st = static_cast<cudaStream_t>(d->cuda_stream);
  e = cudaMemsetAsync(&s->counter, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) {
    k_noalloc_minmax<<<(unsigned)blocks, kThreads, 0, st>>>(eps_real_dev, N, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(&s->counter, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) {
    k_noalloc_maxdev<<<(unsigned)blocks, kThreads, 0, st>>>(eps_real_dev, N, L, s);
    e = cudaGetLastError();
  }
  double res[2] = {0, 0};
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, &s->k0sq, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, &s->bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return err(CBS_ERR_CUDA, "splitting kernels failed: %s", cudaGetErrorString(e));
  if (bad) return err(CBS_ERR_ARG, "permittivity contains a non-finite value");
  if (!(res[1] > 0.0) || !std::isfinite(res[1]))
    return err(CBS_ERR_ARG, "epsilon = %g: a lossless homogeneous grid has no convergent splitting", res[1]);
  const double sc = 1.0 / (d->pitch_m * d->pitch_m);
  *k0sq = res[0] * sc;
  *epsilon = res[1] * sc;
  return CBS_OK;
}
