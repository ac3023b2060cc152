// yz_kernels.cuh -- the strided passes of one CBS iteration, fed by the Tensor Memory Accelerator.
//
//   y pass:  W_c <- FFT_y(W_c) or IFFT_y(W_c), one (component, z) plane x TX columns per tile
//   z pass:  W <- IFFT_z( G(p) FFT_z(W) ), the three components of one y row x TX columns,
//            where G(p) = (I - p p^T / kt2) / (|p|^2 - kt2), kt2 = k0^2 + i epsilon, is the
//            dyadic Green's function of curl curl - kt2 (the vector CBS of refs. [25], [26] of
//            arXiv 2506.15411), scaled by 1/N for the inverse FFT (Nyquist treatment at green()).
//
// Forward transforms are in-place decimation in frequency and leave each axis' spectrum in
// digit-reversed order in W; inverse transforms are decimation in time and restore natural
// order (fft_ip.cuh).  So the y rows the z pass sees are y frequencies in that order, and the
// k-space multiply takes each position's wave number from the per-axis tables.  In the z pass
// the last forward stage, the multiply and the first inverse stage run on the same values in
// registers.
//
// A tile arrives by a few cp.async.bulk.tensor copies (boxes of TX columns x up to 64 rows;
// rows past the end of an axis are zero-filled and never stored), is transformed in place in
// shared memory and leaves by tensor stores.  A block is persistent and keeps nbuf tile
// buffers: while it transforms tile i, the copies of tiles i+1 .. i+nbuf-1 are in flight.  The
// workspace W has a padded row pitch (nxp, a multiple of 16 complex values) so that every
// tensor stride is a multiple of 16 bytes and every box row starts on a 128-byte boundary.
#pragma once
#include <algorithm>

#include "cbs_internal.h"
#include "fft_ip.cuh"
#include "tma.cuh"

namespace cbs {

namespace yzk {

// k-space multiply at wave vector p (q = p except 0 in a Nyquist component):
//   X <- [X + q (q.X) / (|p|^2 - |q|^2 - kt2)] * invN / (|p|^2 - kt2),
// the inverse of |p|^2 I - q q^T - kt2 I.  A Nyquist component (even axis length, wave number
// pi/pitch whose sign is undefined) is 0 in q, which keeps the discrete curl curl real and
// symmetric.  Away from Nyquist q = p and this is (I - p p^T / kt2) / (|p|^2 - kt2).
__device__ __forceinline__ void green(float px, float py, float pz, float qx, float qy, float qz, float2 kt2,
                                      float invN, float2& X0, float2& X1, float2& X2) {
  const float p2 = px * px + py * py + pz * pz;
  const float nyq2 = (px * px - qx * qx) + (py * py - qy * qy) + (pz * pz - qz * qz);
  const float cr = nyq2 - kt2.x, ci = -kt2.y;
  const float cs = __fdividef(1.0f, cr * cr + ci * ci);
  const float2 qd = make_float2(qx * X0.x + qy * X1.x + qz * X2.x, qx * X0.y + qy * X1.y + qz * X2.y);
  const float2 c = cmul(qd, make_float2(cr * cs, -ci * cs));
  const float dr = p2 - kt2.x, di = -kt2.y;
  const float sc = invN * __fdividef(1.0f, dr * dr + di * di);
  const float2 inv = make_float2(dr * sc, -di * sc);   // invN / (dr + i di)
  X0 = cmul(make_float2(X0.x + qx * c.x, X0.y + qx * c.y), inv);
  X1 = cmul(make_float2(X1.x + qy * c.x, X1.y + qy * c.y), inv);
  X2 = cmul(make_float2(X2.x + qz * c.x, X2.y + qz * c.y), inv);
}

#ifndef CBS_Y_THREADS
#define CBS_Y_THREADS 512
#endif
#ifndef CBS_Y2_THREADS
#define CBS_Y2_THREADS 256
#endif
#ifndef CBS_Z_THREADS
#define CBS_Z_THREADS 512
#endif
#ifndef CBS_Z_OCC
#define CBS_Z_OCC 1
#endif
constexpr int kYThreads = CBS_Y_THREADS;    // threads of a y block at one block per SM
constexpr int kY2Threads = CBS_Y2_THREADS;  // ... and at two blocks per SM
constexpr int kZThreads = CBS_Z_THREADS;    // threads of a z block
constexpr int kZOcc = CBS_Z_OCC;            // z blocks per SM

template <int OCC>
constexpr int y_threads() { return OCC == 1 ? kYThreads : kY2Threads; }

// Stages q0 .. q1-1 (forward) or q1-1 .. q0 (inverse) of column transforms of NCOMP x NCOL
// columns held in `buf`, a barrier after each; `after_first` runs after the first barrier.
// PAIRS: butterflies on column pairs (16-byte accesses) or, in the 64-register kernels, on
// single columns.
struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

template <bool INV, int NCOL, int NCOMP, int MAXR, bool PAIRS, class Hook, class Sync = BlockSync>
__device__ __forceinline__ void col_stages(float2* buf, int cs, const AxisIP& ap, int q0, int q1, const float2* tw,
                                           int tid, int nth, Hook after_first, Sync sync = Sync{}) {
  const int ns = ap.ns;
  for (int i = 0; i < q1 - q0; ++i) {
    const int q = INV ? q1 - 1 - i : q0 + i;
    const IPStage s = ip_decode_stage(ap, q);
    radix_dispatch<MAXR>(s.R, [&](auto Ri) {
      constexpr int R = decltype(Ri)::value;
      if constexpr (PAIRS) {
        if (q < ns - 1)
          ipc_stage<R, INV, NCOL, NCOMP, true>(buf, cs, s, tw, tid, nth);
        else
          ipc_stage<R, INV, NCOL, NCOMP, false>(buf, cs, s, tw, tid, nth);
      } else {
        if (q < ns - 1)
          ipc_stage1<R, INV, NCOL, NCOMP, true>(buf, cs, s, tw, tid, nth);
        else
          ipc_stage1<R, INV, NCOL, NCOMP, false>(buf, cs, s, tw, tid, nth);
      }
    });
    sync();
    if (i == 0) after_first();
  }
}

// Persistent y pass: block b of a request's grid of G blocks walks the request's tiles
// t = b, b + G, ... through nbuf tile buffers.  Tile i is transformed in buffer i mod nbuf; after its first stage, thread 0 issues
// the copies of tile i + nbuf - 1 into the buffer of tile i - 1 (once that tile's store has
// been read out of it).  OCC blocks per SM: 1 (512 threads, up to 128 registers, all radices)
// or 2 (256 threads each, radices up to MAXR = 11; two independent blocks keep issuing while
// the other waits at a barrier).
template <int TX, bool INV, int OCC>
__global__ void __launch_bounds__(y_threads<OCC>(), OCC) k_ypass(const __grid_constant__ CUtensorMap tm,
                                                                const IterArgs a) {
  constexpr int MAXR = OCC == 1 ? 16 : 11;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tileN = a.nyr * TX, nbuf = a.nbuf_y;
  float2* buf0 = reinterpret_cast<float2*>(smem_raw);   // nbuf x [nyr][TX]
  float2* tw = buf0 + nbuf * tileN;                      // twiddles of the y axis
  uint64_t* full = reinterpret_cast<uint64_t*>(tw + a.twby / sizeof(float2));   // [nbuf]
  int* fail = reinterpret_cast<int*>(full + nbuf);
  const int nxt = (a.nx + TX - 1) / TX;
  const int ntiles = nxt * a.nz * 3;
  const int B = a.yb, nbox = a.nyr / B;
  const uint32_t tile_bytes = (uint32_t)(nbox * B * TX * sizeof(float2));
  const int G = a.grid_y;
  const MemberBlock mb = member_block(blockIdx.x, G);
  const int c0 = 3 * a.mem[mb.j].seat;   // the request's first component in the tensor map
  if (mb.b >= ntiles) return;
  if (!block_setup_n(buf0, full, nbuf, fail, a.err)) return;
  auto issue = [&](int tt, int bb, uint32_t extra) {
    mbar_arrive_expect_tx(&full[bb], tile_bytes + extra);
    const int xt = tt % nxt, r = tt / nxt;
    const int z = r % a.nz, c = r / a.nz;
    for (int b = 0; b < nbox; ++b)
      tma_load_5d(buf0 + bb * tileN + b * B * TX, &tm, xt * TX, 0, z, b, c0 + c, &full[bb]);
  };
  const int tid = threadIdx.x, nth = blockDim.x;
  if (tid == 0) {
    issue(mb.b, 0, a.twby);   // the first tile's barrier also counts the twiddles
    bulk_load(tw, a.twy, a.twby, &full[0]);
    for (int d = 1; d < nbuf - 1; ++d)
      if (mb.b + d * G < ntiles) issue(mb.b + d * G, d, 0);
  }
  int b = 0;
  for (int i = 0, t = mb.b; t < ntiles; ++i, t += G, b = (b + 1 == nbuf) ? 0 : b + 1) {
    float2* cur = buf0 + b * tileN;
    if (!block_wait(&full[b], fail, a.err, (uint32_t)((i / nbuf) & 1))) return;
    auto prefetch = [&] {
      const int tn = t + (nbuf - 1) * G;
      if (tid == 0 && tn < ntiles) {
        bulk_wait_read_all();   // the store of tile i - 1 has left the buffer
        issue(tn, b == 0 ? nbuf - 1 : b - 1, 0);
      }
    };
    // paired butterflies when the block has 128 registers a thread, single ones at 64
    col_stages<INV, TX, 1, MAXR, y_threads<OCC>() * OCC <= 512>(cur, 0, a.ay, 0, a.ay.ns, tw, tid, nth, prefetch);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      const int xt = t % nxt, r = t / nxt;
      const int z = r % a.nz, c = r / a.nz;
      for (int bx = 0; bx < nbox; ++bx) tma_store_5d(&tm, xt * TX, 0, z, bx, c0 + c, cur + bx * B * TX);
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait_all();
}

// Bar.sync on named barrier `id` (1..15) for `count` threads: the barrier of one warp group.
__device__ __forceinline__ void group_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Persistent z pass (same pipeline as the y pass, one block per SM): forward stages 0 .. s-2
// of the three components of a tile, the fused last forward stage + k-space multiply + first
// inverse stage (single columns, 3 R values in registers; the z wave numbers come from shared
// memory, the x and y ones from the global tables), inverse stages s-2 .. 0.
// The block's threads form a.zgroups (1 or 2) warp groups with their own named barriers; group
// g takes the block's tiles i = g, g + zgroups, ..., so that while one group waits at a barrier
// the other computes.  Tile i sits in buffer i mod nbuf; after its first stage, a group's leader
// issues the copies of tile i + D (D = nbuf - zgroups) into the buffer of the group's own
// previous tile, once that tile's store has been read out of it (a thread can only wait for
// the bulk copies it committed itself).  Tiles 0 .. D-1 are issued up front; the twiddle and
// wave-number tables have their own barrier.
template <int TX, int MAXR>
__global__ void __launch_bounds__(kZThreads, kZOcc) k_zpass_green(const __grid_constant__ CUtensorMap tm,
                                                               const IterArgs a) {
  static_assert(kZThreads % (2 * TX) == 0, "a warp group's threads must be a multiple of the tile width");
  const int NG = a.zgroups, GT = kZThreads / NG;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int nzr = a.nzr;
  const int cs = nzr * TX, tileN = 3 * cs, nbuf = a.nbuf_z;
  float2* buf0 = reinterpret_cast<float2*>(smem_raw);   // nbuf x [3][nzr][TX]
  float2* tw = buf0 + nbuf * tileN;                      // twiddles of the z axis
  float2* pqz = tw + a.twbz / sizeof(float2);            // wave numbers of the z positions
  uint64_t* full = reinterpret_cast<uint64_t*>(pqz + a.pqbz / sizeof(float2));   // [nbuf], then tables
  uint64_t* tbar = full + nbuf;
  int* fail = reinterpret_cast<int*>(tbar + 1);          // [NG] (8 bytes)
  const int nxt = (a.nx + TX - 1) / TX;
  const int ntiles = nxt * a.ny;
  const int B = a.zb, nbox = nzr / B;
  const uint32_t tile_bytes = (uint32_t)(3 * nbox * B * TX * sizeof(float2));
  const int G = a.grid_z;
  const MemberBlock mb = member_block(blockIdx.x, G);
  const int c0 = 3 * a.mem[mb.j].seat;   // the request's first component in the tensor map
  const float2 kt2 = a.mem[mb.j].kt2;
  if (mb.b >= ntiles) return;
  const int tid = threadIdx.x, g = tid / GT, lt = tid - g * GT;
  if (tid == 0) fail[1] = 0;
  if (!block_setup_n(buf0, full, nbuf + 1, fail, a.err)) return;   // also clears fail[0]
  auto issue = [&](int tt, int bb) {
    mbar_arrive_expect_tx(&full[bb], tile_bytes);
    const int xt = tt % nxt, y = tt / nxt;
    const int yb = y / a.yblk, yi = y - yb * a.yblk;
    for (int c = 0; c < 3; ++c)
      for (int b = 0; b < nbox; ++b)
        tma_load_5d(buf0 + bb * tileN + (c * nzr + b * B) * TX, &tm, xt * TX, yi, b * B, yb, c0 + c, &full[bb]);
  };
  const int D = nbuf - NG;   // prefetch distance in tiles
  if (tid == 0) {
    mbar_arrive_expect_tx(tbar, a.twbz + a.pqbz);
    bulk_load(tw, a.twz, a.twbz, tbar);
    bulk_load(pqz, a.pqz, a.pqbz, tbar);
    for (int d = 0; d < D; ++d)
      if (mb.b + d * G < ntiles) issue(mb.b + d * G, d);
  }
  auto gsync = [&] {
    if (NG == 1) __syncthreads();
    else group_sync(1 + g, GT);
  };
  // bounded wait of the group on an mbarrier phase; a timeout aborts the group uniformly
  auto gwait = [&](uint64_t* bar, uint32_t parity) {
    if (!mbar_wait(bar, parity)) fail[g] = 1;
    gsync();
    if (fail[g]) {
      if (lt == 0) atomicExch(a.err, kErrTmaTimeout);
      return false;
    }
    return true;
  };
  if (!gwait(tbar, 0)) return;
  const int ns = a.az.ns;
  const IPStage sl = ip_decode_stage(a.az, ns - 1);
  for (int i = g, t = mb.b + g * G; t < ntiles; i += NG, t += NG * G) {
    const int b = i % nbuf;
    float2* cur = buf0 + b * tileN;
    if (!gwait(&full[b], (uint32_t)((i / nbuf) & 1))) return;
    auto prefetch = [&] {
      const int tn = t + D * G;
      if (lt == 0 && tn < ntiles) {
        bulk_wait_read_all();   // this group's store of tile i - NG has left the buffer
        issue(tn, (i + D) % nbuf);
      }
    };
    const int xt = t % nxt, y = t / nxt;
    const int x0 = xt * TX;
    const float2 pqy = __ldg(&a.pqy[y]);
    // the fused stage gives thread lt the items lt, lt + GT, ...: all in column lt mod TX, as
    // GT is a multiple of TX; so its x wave number is read once per tile (the table is padded
    // past nx)
    const float2 px = __ldg(&a.pqx[x0 + lt % TX]);
    col_stages<false, TX, 3, MAXR, true>(cur, cs, a.az, 0, ns - 1, tw, lt, GT, prefetch, gsync);
    radix_dispatch<MAXR>(sl.R, [&](auto Ri) {
      constexpr int R = decltype(Ri)::value;
      ipz_fused<R, TX>(cur, cs, sl, lt, GT, [&](int, int pos, float2& X0, float2& X1, float2& X2) {
        const float2 pz = pqz[pos];
        green(px.x, pqy.x, pz.x, px.y, pqy.y, pz.y, kt2, a.invN, X0, X1, X2);
      });
    });
    gsync();
    if (ns == 1) prefetch();
    col_stages<true, TX, 3, MAXR, true>(cur, cs, a.az, 0, ns - 1, tw, lt, GT, NoHookIP{}, gsync);
    fence_async_smem();
    gsync();
    if (lt == 0) {
      const int yb = y / a.yblk, yi = y - yb * a.yblk;
      for (int c = 0; c < 3; ++c)
        for (int bb = 0; bb < nbox; ++bb)
          tma_store_5d(&tm, x0, yi, bb * B, yb, c0 + c, cur + (c * nzr + bb * B) * TX);
      bulk_commit();
    }
  }
  if (lt == 0) bulk_wait_all();
}

}  // namespace yzk

// nbuf tiles + twiddles (+ z wave numbers) + mbarriers (8 bytes each) + 8 bytes for the
// failure flag
inline size_t ypass_smem(const IterArgs& a) {
  return (size_t)a.nbuf_y * a.nyr * a.tx_y * sizeof(float2) + a.twby + 8 * a.nbuf_y + 8;
}
inline size_t zpass_smem(const IterArgs& a) {
  return (size_t)3 * a.nbuf_z * a.nzr * a.tx_z * sizeof(float2) + a.twbz + a.pqbz + 8 * (a.nbuf_z + 1) + 8;
}

// Host side of the kernels of one tile width TX, compiled in their own translation unit
// (ypass_tx*.cu, zpass_tx*.cu) so that the library builds in parallel.
template <int TX>
cudaError_t y_occupancy(const IterArgs& a, int* occ) {
  if (a.occ_y == 2)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, yzk::k_ypass<TX, false, 2>, yzk::kY2Threads,
                                                         ypass_smem(a));
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, yzk::k_ypass<TX, false, 1>, yzk::kYThreads, ypass_smem(a));
}
template <int TX>
cudaError_t y_launch(const CUtensorMap& tm, const IterArgs& a, bool inverse, cudaStream_t s) {
  const size_t sm = ypass_smem(a);
  if (a.occ_y == 2) {
    if (inverse) yzk::k_ypass<TX, true, 2><<<a.grid_y * a.nmem, yzk::kY2Threads, sm, s>>>(tm, a);
    else yzk::k_ypass<TX, false, 2><<<a.grid_y * a.nmem, yzk::kY2Threads, sm, s>>>(tm, a);
  } else {
    if (inverse) yzk::k_ypass<TX, true, 1><<<a.grid_y * a.nmem, yzk::kYThreads, sm, s>>>(tm, a);
    else yzk::k_ypass<TX, false, 1><<<a.grid_y * a.nmem, yzk::kYThreads, sm, s>>>(tm, a);
  }
  return cudaGetLastError();
}
template <int TX>
cudaError_t y_set_smem(int bytes) {
  cudaError_t e = cudaSuccess;
  for (const void* f : {(const void*)yzk::k_ypass<TX, false, 1>, (const void*)yzk::k_ypass<TX, true, 1>,
                        (const void*)yzk::k_ypass<TX, false, 2>, (const void*)yzk::k_ypass<TX, true, 2>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

// The z kernels are compiled per largest radix (8, 11 or 16): the fused stage holds 3 R values
// a thread, so a kernel built for the plan's radices needs fewer registers than one for 16.
template <int TX, class F>
cudaError_t z_with_maxr(int maxr, F&& f) {
  if (maxr <= 8) return f(yzk::k_zpass_green<TX, 8>);
  if (maxr <= 11) return f(yzk::k_zpass_green<TX, 11>);
  return f(yzk::k_zpass_green<TX, 16>);
}
template <int TX>
cudaError_t z_occupancy(const IterArgs& a, int* occ) {
  return z_with_maxr<TX>(a.maxr_z, [&](auto k) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, yzk::kZThreads, zpass_smem(a));
  });
}
template <int TX>
cudaError_t z_launch(const CUtensorMap& tm, const IterArgs& a, cudaStream_t s) {
  return z_with_maxr<TX>(a.maxr_z, [&](auto k) {
    k<<<a.grid_z * a.nmem, yzk::kZThreads, zpass_smem(a), s>>>(tm, a);
    return cudaGetLastError();
  });
}
template <int TX>
cudaError_t z_set_smem(int bytes) {
  cudaError_t e = cudaSuccess;
  for (const void* f : {(const void*)yzk::k_zpass_green<TX, 8>, (const void*)yzk::k_zpass_green<TX, 11>,
                        (const void*)yzk::k_zpass_green<TX, 16>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

#define CBS_YZ_FUNCS(PFX, TX)                                                          \
  PFX template cudaError_t y_occupancy<TX>(const IterArgs&, int*);                     \
  PFX template cudaError_t y_launch<TX>(const CUtensorMap&, const IterArgs&, bool, cudaStream_t); \
  PFX template cudaError_t y_set_smem<TX>(int);
#define CBS_Z_FUNCS(PFX, TX)                                                           \
  PFX template cudaError_t z_occupancy<TX>(const IterArgs&, int*);                     \
  PFX template cudaError_t z_launch<TX>(const CUtensorMap&, const IterArgs&, cudaStream_t); \
  PFX template cudaError_t z_set_smem<TX>(int);

}  // namespace cbs
