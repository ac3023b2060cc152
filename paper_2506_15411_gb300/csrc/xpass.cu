// xpass.cu -- the two passes along x (contiguous rows) of one CBS iteration.
//
//   forward:  W_c = FFT_x(V E_c + S_c)                       (scattering potential and source
//                                                              applied in shared memory)
//   inverse:  W_c = IFFT_x(W_c);  delta_c = gamma (E_c - W_c);  E_c -= delta_c;
//             sum |delta|^2 in FP64                           (update of the preconditioned
//                                                              series, refs. [25], [26] of
//                                                              arXiv 2506.15411)
// A block owns a tile of `rpb` consecutive rows (z, y) of all three components.  Its rows are
// contiguous in the padded layouts of E, V and W (row pitch nxp, 16 complex values), so the
// tile arrives with one bulk copy (cp.async.bulk) per array and component and leaves the same
// way; the transforms run in shared memory with the ping-pong Stockham engine.
#include "stockham.cuh"
#include "tma.cuh"

namespace cbs {

namespace {

__device__ __forceinline__ float2 source_at(const IterArgs& a, int c, int z, int y, int x) {
  const SourceArgs& s = a.src;
  if (s.kind == 0) {
    if (z == s.zp) return s.amp[c];
  } else if (s.kind == 1) {
    if (z == s.pz && y == s.py && x == s.px) return s.amp_dev ? s.amp_dev[c] : s.amp[c];
  } else {
    const size_t idx = ((size_t)z * a.ny + y) * a.nx + x;   // the caller's dense layout
    return cscale(__ldg(&s.user[c * a.N + idx]), s.user_scale);
  }
  return make_float2(0.f, 0.f);
}

// Block reduction of the per-thread residual in FP64, then a last-block-done pass that sums
// the per-block partials in a fixed order into hist[slot] (deterministic).
__device__ __forceinline__ void residual_finish(float acc, const IterArgs& a, double* wsum, int* lastflag) {
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
    *lastflag = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!*lastflag) return;
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

constexpr int kThreads = 256;

// Shared-memory layout of the x tiles: arrays of [3][rpb][nxp] (or [rpb][nxp] for V) complex,
// then the mbarrier, the failure flag, the last-block flag and the warp sums.
struct XTile {
  float2* in;    // forward: E tile;  inverse: W tile
  float2* e;     // inverse: E tile
  float2* v;     // V tile
  float2* scr;   // scratch [3][rpb][nxp]
  float2* tw;    // twiddle table of the x axis
  uint64_t* bar;
  int* fail;
  int* last;
  double* wsum;
};

__device__ __forceinline__ XTile carve(unsigned char* base, int rpb, int nxp, int twb, bool inverse) {
  const int span = rpb * nxp;
  float2* p = reinterpret_cast<float2*>(base);
  XTile t;
  t.in = p;
  p += 3 * span;
  t.e = nullptr;
  if (inverse) {
    t.e = p;
    p += 3 * span;
  }
  t.v = p;
  p += span;
  t.scr = p;
  p += 3 * span;
  t.tw = p;
  p += twb / sizeof(float2);
  t.bar = reinterpret_cast<uint64_t*>(p);
  t.fail = reinterpret_cast<int*>(t.bar + 1);
  t.last = t.fail + 1;
  t.wsum = reinterpret_cast<double*>(t.bar + 2);
  return t;
}

__global__ void __launch_bounds__(kThreads) k_xpass_fwd(const IterArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int rpb = a.rpb, nxp = a.nxp, n = a.nx;
  const int r0 = blockIdx.x * rpb;
  const int nr = min(rpb, a.ny * a.nz - r0);
  const int span = rpb * nxp;
  XTile t = carve(smem_raw, rpb, nxp, a.twbx, false);
  if (!block_setup(t.in, t.bar, t.fail, a.err)) return;
  const uint32_t bytes = (uint32_t)(nr * nxp * sizeof(float2));
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(t.bar, 4 * bytes + a.twbx);
    for (int c = 0; c < 3; ++c) bulk_load(t.in + c * span, a.E + c * a.Nw + (size_t)r0 * nxp, bytes, t.bar);
    bulk_load(t.v, a.V + (size_t)r0 * nxp, bytes, t.bar);
    bulk_load(t.tw, a.twx, a.twbx, t.bar);
  }
  if (!block_wait(t.bar, t.fail, a.err)) return;
  const int tid = threadIdx.x, nth = blockDim.x;
  // V E + S in place (the row padding stays as loaded: zeros)
  for (int k = tid; k < 3 * nr * n; k += nth) {
    const int c = k / (nr * n);
    const int rem = k - c * nr * n;
    const int row = rem / n, x = rem - row * n;
    const int gr = r0 + row;
    const int z = gr / a.ny, y = gr - z * a.ny;
    float2& e = t.in[c * span + row * nxp + x];
    e = cadd(cmul(t.v[row * nxp + x], e), source_at(a, c, z, y, x));
  }
  __syncthreads();
  const float2* w = fft_rows<false>(t.in, t.scr, nr, 3, nxp, span, a.ax, t.tw, tid, nth);
  fence_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < 3; ++c) bulk_store(a.W + c * a.Nw + (size_t)r0 * nxp, w + c * span, bytes);
    bulk_commit();
    bulk_wait_all();
  }
}

__global__ void __launch_bounds__(kThreads) k_xpass_inv_update(const IterArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int rpb = a.rpb, nxp = a.nxp, n = a.nx;
  const int r0 = blockIdx.x * rpb;
  const int nr = min(rpb, a.ny * a.nz - r0);
  const int span = rpb * nxp;
  XTile t = carve(smem_raw, rpb, nxp, a.twbx, true);
  if (!block_setup(t.in, t.bar, t.fail, a.err)) return;
  const uint32_t bytes = (uint32_t)(nr * nxp * sizeof(float2));
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(t.bar, 7 * bytes + a.twbx);
    bulk_load(t.tw, a.twx, a.twbx, t.bar);
    for (int c = 0; c < 3; ++c) {
      bulk_load(t.in + c * span, a.W + c * a.Nw + (size_t)r0 * nxp, bytes, t.bar);
      bulk_load(t.e + c * span, a.E + c * a.Nw + (size_t)r0 * nxp, bytes, t.bar);
    }
    bulk_load(t.v, a.V + (size_t)r0 * nxp, bytes, t.bar);
  }
  if (!block_wait(t.bar, t.fail, a.err)) return;
  const int tid = threadIdx.x, nth = blockDim.x;
  const float2* w = fft_rows<true>(t.in, t.scr, nr, 3, nxp, span, a.ax, t.tw, tid, nth);
  const float ie = a.inv_eps;
  float acc = 0.f;
  for (int k = tid; k < nr * n; k += nth) {
    const int row = k / n, x = k - row * n;
    const int o = row * nxp + x;
    const float2 v = t.v[o];
    const float2 g = make_float2(-v.y * ie, v.x * ie);   // gamma = (i / epsilon) V
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 e = t.e[c * span + o];
      const float2 d = cmul(g, csub(e, w[c * span + o]));
      t.e[c * span + o] = csub(e, d);
      acc = fmaf(d.x, d.x, fmaf(d.y, d.y, acc));
    }
  }
  fence_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < 3; ++c) bulk_store(a.E + c * a.Nw + (size_t)r0 * nxp, t.e + c * span, bytes);
    bulk_commit();
  }
  residual_finish(acc, a, t.wsum, t.last);
  if (threadIdx.x == 0) bulk_wait_all();
}

}  // namespace

// tiles, scratch, twiddles, then 8 (mbarrier) + 8 (two flags) + 32 * 8 (warp sums) bytes
size_t xpass_smem(const IterArgs& a) {
  return (size_t)10 * a.rpb * a.nxp * sizeof(float2) + a.twbx + 16 + 32 * 8;
}
size_t xpass_fwd_smem(const IterArgs& a) {
  return (size_t)7 * a.rpb * a.nxp * sizeof(float2) + a.twbx + 16 + 32 * 8;
}
int xpass_blocks(const IterArgs& a) { return (a.ny * a.nz + a.rpb - 1) / a.rpb; }

cudaError_t launch_xpass_fwd(const IterArgs& a, cudaStream_t s) {
  k_xpass_fwd<<<xpass_blocks(a), kThreads, xpass_fwd_smem(a), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_xpass_inv_update(const IterArgs& a, cudaStream_t s) {
  k_xpass_inv_update<<<xpass_blocks(a), kThreads, xpass_smem(a), s>>>(a);
  return cudaGetLastError();
}

cudaError_t xpass_set_smem_limit(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_xpass_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_xpass_inv_update, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace cbs
