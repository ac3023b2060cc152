// xpass.cu -- the passes along x (contiguous rows) of the CBS iterations.
//
//   forward:  W_c = FFT_x(V E_c + S_c)                       (scattering potential and source
//                                                              applied as the first FFT stage
//                                                              loads each element)
//   inverse + next forward (one kernel):
//             W_c = IFFT_x(W_c);  delta_c = gamma (E_c - W_c);  E_c -= delta_c;
//             sum |delta|^2 in FP64, the update applied as the last inverse stage produces
//             each element (update of the preconditioned series, refs. [25], [26] of
//             arXiv 2506.15411); then W_c = FFT_x(V E_c + S_c) of the next iteration from
//             the E just updated, while the tile is still on chip
// A block owns a tile of `rpb` consecutive rows (z, y) of all three components.  Its rows are
// contiguous in the padded layouts of E, V and W (row pitch nxp, 16 complex values), so the
// tile arrives with one bulk copy (cp.async.bulk) per array and component and leaves the same
// way; the transforms run in shared memory with the ping-pong Stockham engine.
#include <algorithm>

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

constexpr int kThreads = 512;

// Shared-memory layout of a pipelined x kernel: two buffer sets, each [3][rpb][nxp] of the
// input (E forward, W inverse), [3][rpb][nxp] of E (inverse only), [rpb][nxp] of V and, in
// the forward kernel, its own scratch [3][rpb][nxp] (an odd number of FFT stages leaves the
// result there, to be stored while the other set computes); then the inverse kernel's shared
// scratch, the x twiddles, two mbarriers, flags and warp sums.
struct XTile {
  float2* in0;      // buffer set 0; set 1 starts `set` elements later
  float2* e0;
  float2* v0;
  int set;
  float2* scr;
  float2* tw;
  uint64_t* full;   // [2]
  int* fail;
  int* last;
  double* wsum;
};

__device__ __forceinline__ XTile carve(unsigned char* base, int rpb, int nxp, int twb, bool inverse) {
  const int span = rpb * nxp;
  float2* p = reinterpret_cast<float2*>(base);
  XTile t;
  t.set = 7 * span;
  t.in0 = p;
  t.e0 = inverse ? p + 3 * span : nullptr;
  t.v0 = p + (inverse ? 6 : 3) * span;
  p += 2 * t.set;
  if (inverse) {
    t.scr = p;            // shared by both sets
    p += 3 * span;
  } else {
    t.scr = t.v0 + span;  // set 0's scratch; set k's is t.scr + k * t.set
  }
  t.tw = p;
  p += twb / sizeof(float2);
  t.full = reinterpret_cast<uint64_t*>(p);
  t.fail = reinterpret_cast<int*>(t.full + 2);
  t.last = t.fail + 1;
  t.wsum = reinterpret_cast<double*>(t.full + 3);
  return t;
}

__device__ __forceinline__ int x_tiles(const IterArgs& a) { return (a.ny * a.nz + a.rpb - 1) / a.rpb; }

// Persistent, double-buffered forward x pass: tile i is transformed in one buffer set while
// the bulk copies of tile i+1 land in the other (issued after the first FFT stage, once the
// store of tile i-1 from that set has left shared memory), and the store of tile i drains
// during the next tile.
__global__ void __launch_bounds__(kThreads, 1) k_xpass_fwd(const IterArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int rpb = a.rpb, nxp = a.nxp;
  const int span = rpb * nxp;
  const int rows = a.ny * a.nz, ntiles = x_tiles(a);
  XTile t = carve(smem_raw, rpb, nxp, a.twbx, false);
  int tile = blockIdx.x;
  if (tile >= ntiles) return;
  if (!block_setup_n(t.in0, t.full, 2, t.fail, a.err)) return;
  const int tid = threadIdx.x, nth = blockDim.x;
  const float inv_ny = 1.0f / (float)a.ny;
  auto issue = [&](int tt, int k, uint32_t extra) {
    const int r0 = tt * rpb, nr = min(rpb, rows - r0);
    const uint32_t bytes = (uint32_t)(nr * nxp * sizeof(float2));
    mbar_arrive_expect_tx(&t.full[k], 4 * bytes + extra);
    for (int c = 0; c < 3; ++c) bulk_load(t.in0 + k * t.set + c * span, a.E + c * a.Nw + (size_t)r0 * nxp, bytes, &t.full[k]);
    bulk_load(t.v0 + k * t.set, a.V + (size_t)r0 * nxp, bytes, &t.full[k]);
  };
  if (tid == 0) {
    issue(tile, 0, a.twbx);
    bulk_load(t.tw, a.twx, a.twbx, &t.full[0]);
  }
  for (int i = 0; tile < ntiles; ++i, tile += gridDim.x) {
    const int k = i & 1;
    const int r0 = tile * rpb, nr = min(rpb, rows - r0);
    const int tn = tile + gridDim.x;
    if (!block_wait(&t.full[k], t.fail, a.err, (uint32_t)((i >> 1) & 1))) return;
    float2* in = t.in0 + k * t.set;
    const float2* v = t.v0 + k * t.set;
    // V E + S, formed as the first FFT stage loads each element
    auto pre = [&](int c, int row, int x, float2 e) {
      const int gr = r0 + row;
      const int z = fdiv(gr, inv_ny), y = gr - z * a.ny;
      return cadd(cmul(v[row * nxp + x], e), source_at(a, c, z, y, x));
    };
    auto prefetch = [&] {
      if (tid == 0 && tn < ntiles) {
        bulk_wait_read_all();   // the store of tile i-1 (from set k^1) has left shared memory
        issue(tn, k ^ 1, 0);
      }
    };
    const float2* w = fft_rows<false>(in, t.scr + k * t.set, nr, 3, nxp, span, a.ax, t.tw, tid, nth, pre, NoPost{},
                                      prefetch);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)(nr * nxp * sizeof(float2));
      for (int c = 0; c < 3; ++c) bulk_store(a.W + c * a.Nw + (size_t)r0 * nxp, w + c * span, bytes);
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait_all();
}

// Persistent, double-buffered x pass that ends one iteration and starts the next on each
// tile: the inverse x transform with the update and the FP64 residual, the store of E, then
// the forward x transform of V E + S of the next iteration (formed from the updated E as its
// first stage computes its inputs) and the store of W.  The series' first iteration runs
// k_xpass_fwd before it; after the last one the W it leaves is not used.
__global__ void __launch_bounds__(kThreads, 1) k_xpass_inv_fwd(const IterArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int rpb = a.rpb, nxp = a.nxp;
  const int span = rpb * nxp;
  const int rows = a.ny * a.nz, ntiles = x_tiles(a);
  XTile t = carve(smem_raw, rpb, nxp, a.twbx, true);
  int tile = blockIdx.x;
  float acc = 0.f;
  const int tid = threadIdx.x, nth = blockDim.x;
  if (tile < ntiles) {
    if (!block_setup_n(t.in0, t.full, 2, t.fail, a.err)) return;
    auto issue = [&](int tt, int k, uint32_t extra) {
      const int r0 = tt * rpb, nr = min(rpb, rows - r0);
      const uint32_t bytes = (uint32_t)(nr * nxp * sizeof(float2));
      mbar_arrive_expect_tx(&t.full[k], 7 * bytes + extra);
      for (int c = 0; c < 3; ++c) {
        bulk_load(t.in0 + k * t.set + c * span, a.W + c * a.Nw + (size_t)r0 * nxp, bytes, &t.full[k]);
        bulk_load(t.e0 + k * t.set + c * span, a.E + c * a.Nw + (size_t)r0 * nxp, bytes, &t.full[k]);
      }
      bulk_load(t.v0 + k * t.set, a.V + (size_t)r0 * nxp, bytes, &t.full[k]);
    };
    if (tid == 0) {
      issue(tile, 0, a.twbx);
      bulk_load(t.tw, a.twx, a.twbx, &t.full[0]);
    }
    const float ie = a.inv_eps;
    const float inv_ny = 1.0f / (float)a.ny;
    // the forward transform's ping-pong buffers, ordered so that its result lands in the
    // tile's W buffer (an odd number of stages >= 3 ends in the second one)
    const bool res_in_b = (a.ax.ns % 2 == 1) && a.ax.ns >= 3;
    for (int i = 0; tile < ntiles; ++i, tile += gridDim.x) {
      const int k = i & 1;
      const int r0 = tile * rpb, nr = min(rpb, rows - r0);
      const int tn = tile + gridDim.x;
      if (!block_wait(&t.full[k], t.fail, a.err, (uint32_t)((i >> 1) & 1))) return;
      auto prefetch = [&] {
        if (tid == 0 && tn < ntiles) {
          bulk_wait_read_all();   // the store of tile i-1 (from set k^1) has left shared memory
          issue(tn, k ^ 1, 0);
        }
      };
      float2* e = t.e0 + k * t.set;
      const float2* v = t.v0 + k * t.set;
      // the update, applied as the last inverse-FFT stage produces each W element:
      // delta = gamma (E - W), gamma = (i / epsilon) V; E -= delta; acc += |delta|^2
      auto post = [&](int c, int row, int x, float2 w) {
        const int o = row * nxp + x;
        const float2 vv = v[o];
        const float2 g = make_float2(-vv.y * ie, vv.x * ie);
        const float2 ec = e[c * span + o];
        const float2 d = cmul(g, csub(ec, w));
        e[c * span + o] = csub(ec, d);
        acc = fmaf(d.x, d.x, fmaf(d.y, d.y, acc));
      };
      float2* win = t.in0 + k * t.set;
      fft_rows<true>(win, t.scr, nr, 3, nxp, span, a.ax, t.tw, tid, nth, NoPre{}, post, prefetch);
      fence_async_smem();
      __syncthreads();
      const uint32_t bytes = (uint32_t)(nr * nxp * sizeof(float2));
      if (tid == 0) {
        for (int c = 0; c < 3; ++c) bulk_store(a.E + c * a.Nw + (size_t)r0 * nxp, e + c * span, bytes);
        bulk_commit();
      }
      // next iteration: W = FFT_x(V E + S) from the updated E (read while its store drains)
      auto gen = generate([&](int c, int row, int x) {
        const int gr = r0 + row;
        const int z = fdiv(gr, inv_ny), y = gr - z * a.ny;
        const int o = row * nxp + x;
        return cadd(cmul(v[o], e[c * span + o]), source_at(a, c, z, y, x));
      });
      const float2* w = fft_rows<false>(res_in_b ? t.scr : win, res_in_b ? win : t.scr, nr, 3, nxp, span, a.ax,
                                        t.tw, tid, nth, gen, NoPost{});
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        for (int c = 0; c < 3; ++c) bulk_store(a.W + c * a.Nw + (size_t)r0 * nxp, w + c * span, bytes);
        bulk_commit();
      }
    }
  }
  residual_finish(acc, a, t.wsum, t.last);
  if (tid == 0) bulk_wait_all();
}

}  // namespace

// two buffer sets, scratch, twiddles, then 16 (two mbarriers) + 8 (two flags) + 32 * 8
// (warp sums) bytes
size_t xpass_smem(const IterArgs& a) {
  return (size_t)17 * a.rpb * a.nxp * sizeof(float2) + a.twbx + 24 + 32 * 8;
}
size_t xpass_fwd_smem(const IterArgs& a) {
  return (size_t)14 * a.rpb * a.nxp * sizeof(float2) + a.twbx + 24 + 32 * 8;
}
int xpass_tiles(const IterArgs& a) { return (a.ny * a.nz + a.rpb - 1) / a.rpb; }

// Persistent grids: as many blocks as fit at once (the inverse pass's, which is also the
// number of residual partials), capped by the tile count.
cudaError_t x_grid_size(IterArgs& a, int sms) {
  int occ_f = 0, occ_i = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, k_xpass_fwd, kThreads, xpass_fwd_smem(a));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_i, k_xpass_inv_fwd, kThreads, xpass_smem(a));
  if (e != cudaSuccess) return e;
  a.grid_x = std::max(1, std::min(xpass_tiles(a), sms * std::max(1, occ_i)));
  a.grid_xf = std::max(1, std::min(xpass_tiles(a), sms * std::max(1, occ_f)));
  return cudaSuccess;
}

cudaError_t launch_xpass_fwd(const IterArgs& a, cudaStream_t s) {
  k_xpass_fwd<<<a.grid_xf, kThreads, xpass_fwd_smem(a), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_xpass_inv_fwd(const IterArgs& a, cudaStream_t s) {
  k_xpass_inv_fwd<<<a.grid_x, kThreads, xpass_smem(a), s>>>(a);
  return cudaGetLastError();
}

cudaError_t xpass_set_smem_limit(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_xpass_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_xpass_inv_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace cbs
