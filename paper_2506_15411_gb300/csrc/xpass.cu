// xpass.cu -- the passes along x (contiguous rows) of the CBS iterations.
//
//   forward:  W_c = FFT_x(V E_c + S_c)                       (scattering potential and source
//                                                              formed as the first FFT stage
//                                                              loads each element)
//   inverse + next forward (one kernel):
//             W_c = IFFT_x(W_c);  delta_c = gamma (E_c - W_c);  E_c -= delta_c;
//             sum |delta|^2 in FP64 (the update of the preconditioned series, refs. [25], [26]
//             of arXiv 2506.15411); then W_c = FFT_x(V E_c + S_c) of the next iteration from
//             the E just updated, while the tile is still on chip
// The forward transforms are in-place decimation in frequency (the x spectrum stays in
// digit-reversed order in W), the inverse ones decimation in time (fft_ip.cuh).  In the fused
// kernel the last inverse stage, the update and the first forward stage of the next iteration
// work on the same butterfly's values in registers, so the updated field never waits for a
// barrier before it is transformed again.
// A block owns a tile of `rpb` consecutive rows (z, y) of all three components.  Its rows are
// contiguous in the padded layouts of E, V and W (row pitch nxp, 16 complex values), so the
// tile arrives with one bulk copy (cp.async.bulk) per array and component and leaves the same
// way.  A block is persistent and keeps nset buffer sets: while it works on tile i, the copies
// of tiles i+1 .. i+nset-1 are in flight.
#include <algorithm>

#include "cbs_internal.h"
#include "fft_ip.cuh"
#include "tma.cuh"

namespace cbs {

namespace {

// The source of component c at voxel (x, y, z); kind and plane (the sheet's z, or the point's
// z) are s.kind and s.zp / s.pz, read once into registers by the caller.
__device__ __forceinline__ float2 source_at(const IterArgs& a, const SourceArgs& s, int kind, int plane, int c,
                                            int z, int y, int x) {
  if (kind == 0) {
    if (z == plane) return s.amp[c];
  } else if (kind == 1) {
    if (z == plane && y == s.py && x == s.px) return s.amp_dev ? s.amp_dev[c] : s.amp[c];
  } else {
    const size_t idx = ((size_t)z * a.ny + y) * a.nx + x;   // the caller's dense layout
    return cscale(__ldg(&s.user[c * a.N + idx]), s.user_scale);
  }
  return make_float2(0.f, 0.f);
}

// Block reduction of the per-thread residual in FP64, then a last-block-done pass that sums
// the per-block partials of the request in seat `seat` (blocks b = 0 .. G-1 of its grid) in a
// fixed order into its hist[slot] (deterministic).
__device__ __forceinline__ void residual_finish(float acc, const IterArgs& a, int seat, int b, int G, double* wsum,
                                                int* lastflag) {
  double* const part = a.partials + (size_t)seat * a.grid_x;
  unsigned* const counter = a.counter + seat;
  double d = (double)acc;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  if (lane == 0) wsum[wid] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double bs = 0.0;
    for (int w = 0; w < nw; ++w) bs += wsum[w];
    part[b] = bs;
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    *lastflag = (prev == (unsigned)G - 1);
  }
  __syncthreads();
  if (!*lastflag) return;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < G; i += blockDim.x) s += __ldcg(&part[i]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  __syncthreads();
  if (lane == 0) wsum[wid] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double bs = 0.0;
    for (int w = 0; w < nw; ++w) bs += wsum[w];
    a.hist[(size_t)seat * a.hist_cap + a.slot] = bs;
    *counter = 0u;
  }
}

#ifndef CBS_X_THREADS
#define CBS_X_THREADS 512
#endif
#ifndef CBS_X_OCC
#define CBS_X_OCC 1
#endif
constexpr int kThreads = CBS_X_THREADS;   // threads of an x block (at most 1024: 32 warp sums)
constexpr int kXOcc = CBS_X_OCC;          // x blocks per SM

// Shared-memory layout of an x kernel: nset buffer sets, each NARR arrays of [rpb][nxp]
// (inverse kernel: W of 3 components, E of 3, V; forward kernel: E of 3 -- transformed in
// place into W -- and V), then the x twiddles, nset mbarriers, flags and warp sums.
struct XTile {
  float2* set0;
  int set;          // elements per buffer set
  float2* tw;
  uint64_t* full;   // [nset]
  uint64_t* tbar;   // the twiddle table's copy
  int* fail;        // [2]: per warp group
  int* last;
  double* wsum;
};

__device__ __forceinline__ XTile carve(unsigned char* base, int rpb, int nxp, int twb, int nset, int narr) {
  const int span = rpb * nxp;
  float2* p = reinterpret_cast<float2*>(base);
  XTile t;
  t.set0 = p;
  t.set = narr * span;
  p += nset * t.set;
  t.tw = p;
  p += twb / sizeof(float2);
  t.full = reinterpret_cast<uint64_t*>(p);
  t.tbar = t.full + nset;
  t.fail = reinterpret_cast<int*>(t.tbar + 1);
  t.last = t.fail + 2;
  t.wsum = reinterpret_cast<double*>(t.fail + 4);
  return t;
}

// Named barrier `id` (1..15) for `count` threads: the barrier of one warp group.
__device__ __forceinline__ void group_sync_x(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
struct BlockSyncX {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

__device__ __forceinline__ int x_tiles(const IterArgs& a) { return (a.ny * a.nz + a.rpb - 1) / a.rpb; }

// (y, z) of memory row r of the y-blocked arrays: r = ((y / yblk) nz + z) yblk + y mod yblk
struct RowDecode {
  float inv_blk, inv_nz;
  int blk, nz;
  __device__ __forceinline__ void operator()(int r, int& y, int& z) const {
    const int t = ip_div(r, inv_blk), yi = r - t * blk;
    const int yb = ip_div(t, inv_nz);
    z = t - yb * nz;
    y = yb * blk + yi;
  }
};
__device__ __forceinline__ RowDecode row_decode(const IterArgs& a) {
  return RowDecode{1.0f / (float)a.yblk, 1.0f / (float)a.nz, a.yblk, a.nz};
}

// Row stages q0 .. q1-1 (forward) or q1-1 .. q0 (inverse) on ncomp x nr rows, a barrier after
// each; `after_first` runs after the first barrier.
template <bool INV, int MAXR, class Hook, class Sync = BlockSyncX>
__device__ __forceinline__ void row_stages(float2* buf, int cs, int ld, int nr, const AxisIP& ap, int q0, int q1,
                                           const float2* tw, int tid, int nth, Hook after_first, Sync sync = Sync{}) {
  const int ns = ap.ns;
  for (int i = 0; i < q1 - q0; ++i) {
    const int q = INV ? q1 - 1 - i : q0 + i;
    const IPStage s = ip_decode_stage(ap, q);
    radix_dispatch<MAXR>(s.R, [&](auto Ri) {
      constexpr int R = decltype(Ri)::value;
      if (q < ns - 1)
        ipr_stage<R, INV, true>(buf, cs, ld, nr, 3, s, tw, tid, nth);
      else
        ipr_stage<R, INV, false>(buf, cs, ld, nr, 3, s, tw, tid, nth);
    });
    sync();
    if (i == 0) after_first();
  }
}

// Persistent forward x pass (a series' first iteration): V E + S formed as the first stage
// loads each element, transformed in place in the E buffer, stored as W.
template <int MAXR>
__global__ void __launch_bounds__(kThreads, kXOcc) k_xpass_fwd(const IterArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int rpb = a.rpb, nxp = a.nxp, nset = a.nset_xf;
  const int span = rpb * nxp;
  const int rows = a.ny * a.nz, ntiles = x_tiles(a);
  const int G = a.grid_xf;
  const MemberBlock mb = member_block(blockIdx.x, G);
  const Member& mem = a.mem[mb.j];
  const size_t so = (size_t)mem.seat * 3 * a.Nw;
  const float2* const E = a.E + so;
  float2* const W = a.W + so;
  const float2* const V = a.V + (size_t)mem.seat * a.Nw;
  const int skind = mem.src.kind, splane = skind == 1 ? mem.src.pz : mem.src.zp;
  XTile t = carve(smem_raw, rpb, nxp, a.twbx, nset, 4);
  if (mb.b >= ntiles) return;
  if (!block_setup_n(t.set0, t.full, nset, t.fail, a.err)) return;
  const int tid = threadIdx.x, nth = blockDim.x;
  const RowDecode rowdec = row_decode(a);
  auto issue = [&](int tt, int k, uint32_t extra) {
    const int r0 = tt * rpb, nr = min(rpb, rows - r0);
    const uint32_t bytes = (uint32_t)(nr * nxp * sizeof(float2));
    float2* s = t.set0 + k * t.set;
    mbar_arrive_expect_tx(&t.full[k], 4 * bytes + extra);
    for (int c = 0; c < 3; ++c) bulk_load(s + c * span, E + c * a.Nw + (size_t)r0 * nxp, bytes, &t.full[k]);
    bulk_load(s + 3 * span, V + (size_t)r0 * nxp, bytes, &t.full[k]);
  };
  if (tid == 0) {
    issue(mb.b, 0, a.twbx);
    bulk_load(t.tw, a.twx, a.twbx, &t.full[0]);
    for (int d = 1; d < nset - 1; ++d)
      if (mb.b + d * G < ntiles) issue(mb.b + d * G, d, 0);
  }
  const int ns = a.ax.ns;
  const IPStage s0 = ip_decode_stage(a.ax, 0);
  int k = 0;
  for (int i = 0, tile = mb.b; tile < ntiles; ++i, tile += G, k = (k + 1 == nset) ? 0 : k + 1) {
    const int r0 = tile * rpb, nr = min(rpb, rows - r0);
    if (!block_wait(&t.full[k], t.fail, a.err, (uint32_t)((i / nset) & 1))) return;
    float2* e = t.set0 + k * t.set;
    const float2* v = e + 3 * span;
    auto prefetch = [&] {
      const int tn = tile + (nset - 1) * G;
      if (tid == 0 && tn < ntiles) {
        bulk_wait_read_all();   // the store of tile i - 1 has left its buffer set
        issue(tn, k == 0 ? nset - 1 : k - 1, 0);
      }
    };
    auto gen = [&](int c, int row, int x, float2 ev) {
      const int gr = r0 + row;
      int y, z;
      rowdec(gr, y, z);
      return cadd(cmul(v[row * nxp + x], ev), source_at(a, mem.src, skind, splane, c, z, y, x));
    };
    radix_dispatch<MAXR>(s0.R, [&](auto Ri) {
      constexpr int R = decltype(Ri)::value;
      if (ns > 1)
        ipr_dif_first<R, true>(e, span, nxp, nr, 3, s0, t.tw, tid, nth, gen);
      else
        ipr_dif_first<R, false>(e, span, nxp, nr, 3, s0, t.tw, tid, nth, gen);
    });
    __syncthreads();
    prefetch();
    row_stages<false, MAXR>(e, span, nxp, nr, a.ax, 1, ns, t.tw, tid, nth, NoHookIP{});
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)(nr * nxp * sizeof(float2));
      for (int c = 0; c < 3; ++c) bulk_store(W + c * a.Nw + (size_t)r0 * nxp, e + c * span, bytes);
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait_all();
}

// Persistent x pass that ends one iteration and starts the next on each tile: the inverse x
// stages s-1 .. 1, then (fused, in registers) the last inverse stage, the update with the
// FP64 residual and the first forward stage of V E + S of the next iteration, the store of E,
// the forward stages 1 .. s-1 and the store of W.  The series' first iteration runs
// k_xpass_fwd before it; after the last one the W it leaves is not used.
// The block's threads form a.xgroups (1 or 2) warp groups with their own named barriers; group
// g takes the block's tiles i = g, g + xgroups, ...  Tile i sits in buffer set i mod nset; after
// its first stage a group's leader issues the copies of tile i + D (D = nset - xgroups) into the
// set of the group's own previous tile, once that tile's stores have been read out of it.
// A group whose copy wait times out records the error and stops taking tiles, but still
// joins the block's final residual reduction.
template <int MAXR>
__global__ void __launch_bounds__(kThreads, kXOcc) k_xpass_inv_fwd(const IterArgs a) {
  const int NG = a.xgroups, GT = kThreads / NG;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int rpb = a.rpb, nxp = a.nxp, nset = a.nset_x;
  const int span = rpb * nxp;
  const int rows = a.ny * a.nz, ntiles = x_tiles(a);
  const int G = a.grid_x;
  const MemberBlock mb = member_block(blockIdx.x, G);
  const Member& mem = a.mem[mb.j];
  const size_t so = (size_t)mem.seat * 3 * a.Nw;
  float2* const E = a.E + so;
  float2* const W = a.W + so;
  const float2* const V = a.V + (size_t)mem.seat * a.Nw;
  const int skind = mem.src.kind, splane = skind == 1 ? mem.src.pz : mem.src.zp;
  XTile t = carve(smem_raw, rpb, nxp, a.twbx, nset, 7);
  float acc = 0.f;
  const int tid = threadIdx.x, g = tid / GT, lt = tid - g * GT;
  if (mb.b < ntiles) {
    if (tid == 0) t.fail[1] = 0;
    if (!block_setup_n(t.set0, t.full, nset + 1, t.fail, a.err)) return;   // also clears fail[0]
    auto issue = [&](int tt, int k) {
      const int r0 = tt * rpb, nr = min(rpb, rows - r0);
      const uint32_t bytes = (uint32_t)(nr * nxp * sizeof(float2));
      float2* s = t.set0 + k * t.set;
      mbar_arrive_expect_tx(&t.full[k], 7 * bytes);
      for (int c = 0; c < 3; ++c) {
        bulk_load(s + c * span, W + c * a.Nw + (size_t)r0 * nxp, bytes, &t.full[k]);
        bulk_load(s + (3 + c) * span, E + c * a.Nw + (size_t)r0 * nxp, bytes, &t.full[k]);
      }
      bulk_load(s + 6 * span, V + (size_t)r0 * nxp, bytes, &t.full[k]);
    };
    const int D = nset - NG;   // prefetch distance in tiles
    if (tid == 0) {
      mbar_arrive_expect_tx(t.tbar, a.twbx);
      bulk_load(t.tw, a.twx, a.twbx, t.tbar);
      for (int d = 0; d < D; ++d)
        if (mb.b + d * G < ntiles) issue(mb.b + d * G, d);
    }
    auto gsync = [&] {
      if (NG == 1) __syncthreads();
      else group_sync_x(1 + g, GT);
    };
    auto gwait = [&](uint64_t* bar, uint32_t parity) {
      if (!mbar_wait(bar, parity)) t.fail[g] = 1;
      gsync();
      if (t.fail[g]) {
        if (lt == 0) atomicExch(a.err, kErrTmaTimeout);
        return false;
      }
      return true;
    };
    const float ie = mem.inv_eps;
    const RowDecode rowdec = row_decode(a);
    const int ns = a.ax.ns;
    const IPStage s0 = ip_decode_stage(a.ax, 0);
    bool ok = gwait(t.tbar, 0);
    for (int i = g, tile = mb.b + g * G; ok && tile < ntiles; i += NG, tile += NG * G) {
      const int k = i % nset;
      const int r0 = tile * rpb, nr = min(rpb, rows - r0);
      if (!gwait(&t.full[k], (uint32_t)((i / nset) & 1))) {
        ok = false;
        break;
      }
      float2* w = t.set0 + k * t.set;
      float2* e = w + 3 * span;
      const float2* v = w + 6 * span;
      auto prefetch = [&] {
        const int tn = tile + D * G;
        if (lt == 0 && tn < ntiles) {
          bulk_wait_read_all();   // this group's stores of tile i - NG have left their set
          issue(tn, (i + D) % nset);
        }
      };
      row_stages<true, MAXR>(w, span, nxp, nr, a.ax, 1, ns, t.tw, lt, GT, prefetch, gsync);
      // the update at each natural-order element of the inverse transform, then the input of
      // the next forward transform there:
      //   delta = gamma (E - W), gamma = (i / epsilon) V;  E -= delta;  acc += |delta|^2;
      //   returns V E + S
      auto f = [&](int c, int row, int x, float2 wv) {
        const int o = row * nxp + x;
        const float2 vv = v[o];
        const float2 gm = make_float2(-vv.y * ie, vv.x * ie);
        const float2 ec = e[c * span + o];
        const float2 d = cmul(gm, csub(ec, wv));
        const float2 en = csub(ec, d);
        e[c * span + o] = en;
        acc = fmaf(d.x, d.x, fmaf(d.y, d.y, acc));
        int y, z;
        rowdec(r0 + row, y, z);
        return cadd(cmul(vv, en), source_at(a, mem.src, skind, splane, c, z, y, x));
      };
      radix_dispatch<MAXR>(s0.R, [&](auto Ri) {
        constexpr int R = decltype(Ri)::value;
        if (ns > 1)
          ipx_fused<R, true>(w, span, nxp, nr, 3, s0, t.tw, lt, GT, f);
        else
          ipx_fused<R, false>(w, span, nxp, nr, 3, s0, t.tw, lt, GT, f);
      });
      fence_async_smem();
      gsync();
      if (ns == 1) prefetch();
      const uint32_t bytes = (uint32_t)(nr * nxp * sizeof(float2));
      if (lt == 0) {
        for (int c = 0; c < 3; ++c) bulk_store(E + c * a.Nw + (size_t)r0 * nxp, e + c * span, bytes);
        bulk_commit();
      }
      row_stages<false, MAXR>(w, span, nxp, nr, a.ax, 1, ns, t.tw, lt, GT, NoHookIP{}, gsync);
      fence_async_smem();
      gsync();
      if (lt == 0) {
        for (int c = 0; c < 3; ++c) bulk_store(W + c * a.Nw + (size_t)r0 * nxp, w + c * span, bytes);
        bulk_commit();
      }
    }
  }
  residual_finish(acc, a, mem.seat, mb.b, G, t.wsum, t.last);
  if (lt == 0) bulk_wait_all();
}

}  // namespace

// nset buffer sets of NARR arrays, twiddles, then nset + 1 mbarriers + 16 (flags) + 32 * 8
// (warp sums) bytes
size_t xpass_smem(const IterArgs& a) {
  return (size_t)7 * a.nset_x * a.rpb * a.nxp * sizeof(float2) + a.twbx + 8 * (a.nset_x + 1) + 16 + 32 * 8;
}
size_t xpass_fwd_smem(const IterArgs& a) {
  return (size_t)4 * a.nset_xf * a.rpb * a.nxp * sizeof(float2) + a.twbx + 8 * (a.nset_xf + 1) + 16 + 32 * 8;
}
int xpass_tiles(const IterArgs& a) { return (a.ny * a.nz + a.rpb - 1) / a.rpb; }

template <class F>
cudaError_t with_maxr_x(int maxr, F&& f) {
  if (maxr <= 8) return f(std::integral_constant<int, 8>{});
  if (maxr <= 11) return f(std::integral_constant<int, 11>{});
  return f(std::integral_constant<int, 16>{});
}

// Persistent grids: as many blocks as fit at once (the inverse pass's, which is also the
// number of residual partials), capped by the tile count.
cudaError_t x_grid_size(IterArgs& a, int sms) {
  return with_maxr_x(a.maxr_x, [&](auto M) {
    constexpr int MR = decltype(M)::value;
    int occ_f = 0, occ_i = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, k_xpass_fwd<MR>, kThreads,
                                                                  xpass_fwd_smem(a));
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_i, k_xpass_inv_fwd<MR>, kThreads, xpass_smem(a));
    if (e != cudaSuccess) return e;
    a.grid_x = std::max(1, std::min(xpass_tiles(a), sms * std::max(1, occ_i)));
    a.grid_xf = std::max(1, std::min(xpass_tiles(a), sms * std::max(1, occ_f)));
    return cudaSuccess;
  });
}

cudaError_t launch_xpass_fwd(const IterArgs& a, cudaStream_t s) {
  return with_maxr_x(a.maxr_x, [&](auto M) {
    constexpr int MR = decltype(M)::value;
    k_xpass_fwd<MR><<<a.grid_xf * a.nmem, kThreads, xpass_fwd_smem(a), s>>>(a);
    return cudaGetLastError();
  });
}

cudaError_t launch_xpass_inv_fwd(const IterArgs& a, cudaStream_t s) {
  return with_maxr_x(a.maxr_x, [&](auto M) {
    constexpr int MR = decltype(M)::value;
    k_xpass_inv_fwd<MR><<<a.grid_x * a.nmem, kThreads, xpass_smem(a), s>>>(a);
    return cudaGetLastError();
  });
}

cudaError_t xpass_set_smem_limit(int bytes) {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  };
  set((const void*)k_xpass_fwd<8>);
  set((const void*)k_xpass_fwd<11>);
  set((const void*)k_xpass_fwd<16>);
  set((const void*)k_xpass_inv_fwd<8>);
  set((const void*)k_xpass_inv_fwd<11>);
  set((const void*)k_xpass_inv_fwd<16>);
  return e;
}

}  // namespace cbs
