// yzpass.cu -- the strided passes of one CBS iteration, fed by the Tensor Memory Accelerator.
//
//   y pass:  W_c <- FFT_y(W_c) or IFFT_y(W_c), one (component, z) plane x TX columns per block
//   z pass:  W <- IFFT_z( G(p) FFT_z(W) ), the three components of one y row x TX columns,
//            where G(p) = (I - p p^T / kt2) / (|p|^2 - kt2), kt2 = k0^2 + i epsilon, is the
//            dyadic Green's function of curl curl - kt2 (the vector CBS of refs. [25], [26] of
//            arXiv 2506.15411), scaled by 1/N for the inverse FFT (Nyquist treatment at green()).
//
// A block loads its whole tile with a few cp.async.bulk.tensor copies (boxes of TX columns x
// up to 64 rows; rows past the end of an axis are zero-filled and never stored), transforms it in
// shared memory with the ping-pong Stockham engine, and writes it back with tensor stores.
// The workspace W has a padded row pitch (nxp, a multiple of 16 complex values) so that every
// tensor stride is a multiple of 16 bytes and every box row starts on a 128-byte boundary.
#include <algorithm>

#include "stockham.cuh"
#include "tma.cuh"

namespace cbs {

namespace {

__device__ __forceinline__ int fft_freq(int k, int n) { return (2 * k < n) ? k : k - n; }

// k-space multiply at (kx, ky, kz):
//   X <- [X + q (q.X) / (|p|^2 - |q|^2 - kt2)] * invN / (|p|^2 - kt2),
// the inverse of |p|^2 I - q q^T - kt2 I, where q = p except that a Nyquist component (even
// axis length, wave number pi/pitch whose sign is undefined) is 0 in q, which keeps the
// discrete curl curl real and symmetric.  Away from Nyquist q = p and this is
// (I - p p^T / kt2) / (|p|^2 - kt2).
__device__ __forceinline__ void green(float px, float py, float pz, float qx, float qy, float qz, float2 kt2,
                                      float invN, float2& X0, float2& X1, float2& X2) {
  const float p2 = px * px + py * py + pz * pz;
  const float nyq2 = (px * px - qx * qx) + (py * py - qy * qy) + (pz * pz - qz * qz);
  const float cr = nyq2 - kt2.x, ci = -kt2.y;
  const float cs = __frcp_rn(cr * cr + ci * ci);
  const float2 qd = make_float2(qx * X0.x + qy * X1.x + qz * X2.x, qx * X0.y + qy * X1.y + qz * X2.y);
  const float2 c = cmul(qd, make_float2(cr * cs, -ci * cs));
  const float dr = p2 - kt2.x, di = -kt2.y;
  const float sc = invN * __frcp_rn(dr * dr + di * di);
  const float2 inv = make_float2(dr * sc, -di * sc);   // invN / (dr + i di)
  X0 = cmul(make_float2(X0.x + qx * c.x, X0.y + qx * c.y), inv);
  X1 = cmul(make_float2(X1.x + qy * c.x, X1.y + qy * c.y), inv);
  X2 = cmul(make_float2(X2.x + qz * c.x, X2.y + qz * c.y), inv);
}

constexpr int kYZThreads = 512;

// Persistent, multi-buffered y pass: a block walks tiles t = blockIdx.x, + gridDim.x, ...
// through nbuf tile buffers (3 when they fit, else 2); while it transforms tile i, the tensor
// copies of tile i+1 land in the next buffer (issued after the first FFT stage, once the store
// of the tile that last used that buffer has been read out; with 3 buffers that store was
// issued a whole tile earlier), and the store of tile i drains meanwhile.  Twiddles are
// loaded once.
// OCC blocks per SM: 1 (up to 128 registers, all radices) or 2 (64 registers, radices up to
// MAXR = 11, half the shared memory each; two independent blocks keep issuing while the
// other waits at a barrier).
template <int TX, bool INV, int OCC>
__global__ void __launch_bounds__(kYZThreads, OCC) k_ypass(const __grid_constant__ CUtensorMap tm, const IterArgs a) {
  constexpr int MAXR = OCC == 1 ? 16 : 11;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tileN = a.nyr * TX, nbuf = a.nbuf_y;
  float2* buf0 = reinterpret_cast<float2*>(smem_raw);   // nbuf x [nyr][TX]
  float2* scr = buf0 + nbuf * tileN;                     // [ny][TX]
  float2* tw = scr + a.ny * TX;                          // twiddles of the y axis
  uint64_t* full = reinterpret_cast<uint64_t*>(tw + a.twby / sizeof(float2));   // [nbuf]
  int* fail = reinterpret_cast<int*>(full + nbuf);
  const int nxt = (a.nx + TX - 1) / TX;
  const int ntiles = nxt * a.nz * 3;
  const int B = a.yb, nbox = a.nyr / B;
  const uint32_t tile_bytes = (uint32_t)(nbox * B * TX * sizeof(float2));
  int t = blockIdx.x;
  if (t >= ntiles) return;
  if (!block_setup_n(buf0, full, nbuf, fail, a.err)) return;
  auto issue = [&](int tt, float2* buf, uint64_t* bar) {
    const int xt = tt % nxt, r = tt / nxt;
    const int z = r % a.nz, c = r / a.nz;
    for (int b = 0; b < nbox; ++b) tma_load_4d(buf + b * B * TX, &tm, xt * TX, b * B, z, c, bar);
  };
  const int tid = threadIdx.x, nth = blockDim.x;
  if (tid == 0) {
    mbar_arrive_expect_tx(&full[0], tile_bytes + a.twby);
    bulk_load(tw, a.twy, a.twby, &full[0]);
    issue(t, buf0, &full[0]);
  }
  for (int i = 0, b = 0; t < ntiles; ++i, t += gridDim.x, b = (b + 1 == nbuf) ? 0 : b + 1) {
    float2* cur = buf0 + b * tileN;
    const int bn = (b + 1 == nbuf) ? 0 : b + 1;
    float2* nxb = buf0 + bn * tileN;
    uint64_t* nbar = &full[bn];
    const int tn = t + gridDim.x;
    if (!block_wait(&full[b], fail, a.err, (uint32_t)((i / nbuf) & 1))) return;
    auto prefetch = [&] {
      if (tid == 0 && tn < ntiles) {
        if (nbuf == 2) bulk_wait_read_all();   // the store of tile i-1 has left nxb
        else bulk_wait_read_1();               // all but the newest store (tile i-1) have
        mbar_arrive_expect_tx(nbar, tile_bytes);
        issue(tn, nxb, nbar);
      }
    };
    cols2_stages<INV, TX, 1, MAXR>(cur, cur, scr, 0, a.ay, 0, a.ay.ns, tw, tid, nth, prefetch);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      const int xt = t % nxt, r = t / nxt;
      const int z = r % a.nz, c = r / a.nz;
      for (int b = 0; b < nbox; ++b) tma_store_4d(&tm, xt * TX, b * B, z, c, cur + b * B * TX);
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait_all();
}

// Last forward z stage of the three components of one column (outputs in natural order,
// at the positions it reads), the k-space multiply at its R outputs, written to A.
template <int R, int TX>
__device__ __forceinline__ void stage_last_green(const float2* src, float2* A, int cs, int4 g, const float2* tw,
                                                 int tid, int nth, int x0, float py, float qy, const IterArgs& a) {
  const int stride = g.z, n = a.nz;
  const int items = TX * stride;
  const float two_pi = 6.283185307179586f;
  for (int k = tid; k < items; k += nth) {
    const int col = (int)((unsigned)k % TX), j = (int)((unsigned)k / TX);
    float2 v[3][R];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int r = 0; r < R; ++r) v[c][r] = src[c * cs + (j + r * stride) * TX + col];
    // last stage: Ns = n / R = stride, so j mod Ns = j (j = 0 multiplies by w^0 = 1 exactly)
    if constexpr (R > 1) {
      const int step = j * g.w;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = tw[r * step];
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c][r] = cmul(v[c][r], w);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) DFT<R, false>::run(v[c]);
    const int x = x0 + col;
    const float px = two_pi / (float)a.nx * (float)fft_freq(x, a.nx);
    const float qx = (2 * x == a.nx) ? 0.f : px;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int iz = j + r * stride;
      const float pz = two_pi / (float)n * (float)fft_freq(iz, n);
      const float qz = (2 * iz == n) ? 0.f : pz;
      green(px, py, pz, qx, qy, qz, a.kt2, a.invN, v[0][r], v[1][r], v[2][r]);
#pragma unroll
      for (int c = 0; c < 3; ++c) A[c * cs + iz * TX + col] = v[c][r];
    }
  }
}

// The k-space multiply as its own sweep over a transformed tile (one thread per (z, column)
// point, all three components): the two-blocks-per-SM variant has no registers for the fused
// last stage.
template <int TX>
__device__ __forceinline__ void green_sweep(float2* A, int cs, int x0, float py, float qy, int tid, int nth,
                                            const IterArgs& a) {
  const float two_pi = 6.283185307179586f;
  const float kx = two_pi / (float)a.nx, kz = two_pi / (float)a.nz;
  for (int k = tid; k < TX * a.nz; k += nth) {
    const int col = (int)((unsigned)k % TX), iz = (int)((unsigned)k / TX);
    const int x = x0 + col;
    const float px = kx * (float)fft_freq(x, a.nx);
    const float qx = (2 * x == a.nx) ? 0.f : px;
    const float pz = kz * (float)fft_freq(iz, a.nz);
    const float qz = (2 * iz == a.nz) ? 0.f : pz;
    const int o = iz * TX + col;
    float2 v0 = A[o], v1 = A[cs + o], v2 = A[2 * cs + o];
    green(px, py, pz, qx, qy, qz, a.kt2, a.invN, v0, v1, v2);
    A[o] = v0;
    A[cs + o] = v1;
    A[2 * cs + o] = v2;
  }
}

// Persistent, multi-buffered z pass (same pipeline as the y pass): FFT_z of the three
// components of a tile (their stages run together), the k-space multiply (fused into the last
// forward stage when OCC = 1, a separate sweep when OCC = 2), IFFT_z.
template <int TX, int OCC>
__global__ void __launch_bounds__(kYZThreads, OCC) k_zpass_green(const __grid_constant__ CUtensorMap tm,
                                                                 const IterArgs a) {
  constexpr int MAXR = OCC == 1 ? 16 : 11;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int nzr = a.nzr;
  const int cs = nzr * TX, tileN = 3 * cs, nbuf = a.nbuf_z;
  float2* buf0 = reinterpret_cast<float2*>(smem_raw);   // nbuf x [3][nzr][TX]
  float2* scr = buf0 + nbuf * tileN;                     // [3][nzr][TX]
  float2* tw = scr + tileN;                              // twiddles of the z axis
  uint64_t* full = reinterpret_cast<uint64_t*>(tw + a.twbz / sizeof(float2));   // [nbuf]
  int* fail = reinterpret_cast<int*>(full + nbuf);
  const int nxt = (a.nx + TX - 1) / TX;
  const int ntiles = nxt * a.ny;
  const int B = a.zb, nbox = nzr / B;
  const uint32_t tile_bytes = (uint32_t)(3 * nbox * B * TX * sizeof(float2));
  int t = blockIdx.x;
  if (t >= ntiles) return;
  if (!block_setup_n(buf0, full, nbuf, fail, a.err)) return;
  auto issue = [&](int tt, float2* buf, uint64_t* bar) {
    const int xt = tt % nxt, y = tt / nxt;
    for (int c = 0; c < 3; ++c)
      for (int b = 0; b < nbox; ++b) tma_load_4d(buf + (c * nzr + b * B) * TX, &tm, xt * TX, y, b * B, c, bar);
  };
  const int tid = threadIdx.x, nth = blockDim.x;
  if (tid == 0) {
    mbar_arrive_expect_tx(&full[0], tile_bytes + a.twbz);
    bulk_load(tw, a.twz, a.twbz, &full[0]);
    issue(t, buf0, &full[0]);
  }
  const float two_pi = 6.283185307179586f;
  const int ns = a.az.ns;
  for (int i = 0, b = 0; t < ntiles; ++i, t += gridDim.x, b = (b + 1 == nbuf) ? 0 : b + 1) {
    float2* cur = buf0 + b * tileN;
    const int bn = (b + 1 == nbuf) ? 0 : b + 1;
    float2* nxb = buf0 + bn * tileN;
    uint64_t* nbar = &full[bn];
    const int tn = t + gridDim.x;
    if (!block_wait(&full[b], fail, a.err, (uint32_t)((i / nbuf) & 1))) return;
    auto prefetch = [&] {
      if (tid == 0 && tn < ntiles) {
        if (nbuf == 2) bulk_wait_read_all();
        else bulk_wait_read_1();
        mbar_arrive_expect_tx(nbar, tile_bytes);
        issue(tn, nxb, nbar);
      }
    };
    const int xt = t % nxt, y = t / nxt;
    const int x0 = xt * TX;
    const float py = two_pi / (float)a.ny * (float)fft_freq(y, a.ny);
    const float qy = (2 * y == a.ny) ? 0.f : py;
    if constexpr (OCC == 1) {
      float2* P = cols2_stages<false, TX, 3, MAXR>(cur, cur, scr, cs, a.az, 0, ns - 1, tw, tid, nth, prefetch);
      const int4 g = stage_of(a.az, ns - 1);
      radix_dispatch<MAXR>(g.x, [&](auto Ri) {
        constexpr int R = decltype(Ri)::value;
        stage_last_green<R, TX>(P, cur, cs, g, tw, tid, nth, x0, py, qy, a);
      });
      __syncthreads();
      if (ns == 1) prefetch();
    } else {
      cols2_stages<false, TX, 3, MAXR>(cur, cur, scr, cs, a.az, 0, ns, tw, tid, nth, prefetch);
      green_sweep<TX>(cur, cs, x0, py, qy, tid, nth, a);
      __syncthreads();
    }
    cols2_stages<true, TX, 3, MAXR>(cur, cur, scr, cs, a.az, 0, ns, tw, tid, nth);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      for (int c = 0; c < 3; ++c)
        for (int bb = 0; bb < nbox; ++bb) tma_store_4d(&tm, x0, y, bb * B, c, cur + (c * nzr + bb * B) * TX);
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait_all();
}

template <class F>
cudaError_t with_tx(int tx, F&& f) {
  switch (tx) {
    case 4: return f(std::integral_constant<int, 4>{});
    case 8: return f(std::integral_constant<int, 8>{});
    case 16: return f(std::integral_constant<int, 16>{});
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// nbuf tiles + scratch + twiddles + mbarriers (8 bytes each) + 8 bytes for the failure flag
size_t ypass_smem(const IterArgs& a) {
  return (size_t)(a.nbuf_y * a.nyr + a.ny) * a.tx_y * sizeof(float2) + a.twby + 8 * a.nbuf_y + 8;
}
size_t zpass_smem(const IterArgs& a) {
  return (size_t)3 * (a.nbuf_z + 1) * a.nzr * a.tx_z * sizeof(float2) + a.twbz + 8 * a.nbuf_z + 8;
}
int ypass_tiles(const IterArgs& a) { return (a.nx + a.tx_y - 1) / a.tx_y * a.nz * 3; }
int zpass_tiles(const IterArgs& a) { return (a.nx + a.tx_z - 1) / a.tx_z * a.ny; }

template <class F>
cudaError_t with_occ(int occ, F&& f) {
  return occ == 2 ? f(std::integral_constant<int, 2>{}) : f(std::integral_constant<int, 1>{});
}

// Persistent grids: as many blocks as fit on the device at once (capped by the tile count).
cudaError_t yz_grid_sizes(IterArgs& a, int sms) {
  cudaError_t e = with_tx(a.tx_y, [&](auto T) {
    return with_occ(a.occ_y, [&](auto O) {
      constexpr int TX = decltype(T)::value, OCC = decltype(O)::value;
      int occ = 0;
      cudaError_t e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ypass<TX, false, OCC>, kYZThreads,
                                                                     ypass_smem(a));
      if (e1 == cudaSuccess) a.grid_y = std::max(1, std::min(ypass_tiles(a), sms * std::max(1, occ)));
      return e1;
    });
  });
  if (e != cudaSuccess) return e;
  return with_tx(a.tx_z, [&](auto T) {
    return with_occ(a.occ_z, [&](auto O) {
      constexpr int TX = decltype(T)::value, OCC = decltype(O)::value;
      int occ = 0;
      cudaError_t e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_zpass_green<TX, OCC>, kYZThreads,
                                                                     zpass_smem(a));
      if (e1 == cudaSuccess) a.grid_z = std::max(1, std::min(zpass_tiles(a), sms * std::max(1, occ)));
      return e1;
    });
  });
}

cudaError_t launch_ypass(const CUtensorMap& tm, const IterArgs& a, bool inverse, cudaStream_t s) {
  return with_tx(a.tx_y, [&](auto T) {
    return with_occ(a.occ_y, [&](auto O) {
      constexpr int TX = decltype(T)::value, OCC = decltype(O)::value;
      if (inverse)
        k_ypass<TX, true, OCC><<<a.grid_y, kYZThreads, ypass_smem(a), s>>>(tm, a);
      else
        k_ypass<TX, false, OCC><<<a.grid_y, kYZThreads, ypass_smem(a), s>>>(tm, a);
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_zpass_green(const CUtensorMap& tm, const IterArgs& a, cudaStream_t s) {
  return with_tx(a.tx_z, [&](auto T) {
    return with_occ(a.occ_z, [&](auto O) {
      constexpr int TX = decltype(T)::value, OCC = decltype(O)::value;
      k_zpass_green<TX, OCC><<<a.grid_z, kYZThreads, zpass_smem(a), s>>>(tm, a);
      return cudaGetLastError();
    });
  });
}

cudaError_t yzpass_set_smem_limit(int bytes) {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  };
  auto set_tx = [&](auto T) {
    constexpr int TX = decltype(T)::value;
    set((const void*)k_ypass<TX, false, 1>);
    set((const void*)k_ypass<TX, true, 1>);
    set((const void*)k_ypass<TX, false, 2>);
    set((const void*)k_ypass<TX, true, 2>);
    set((const void*)k_zpass_green<TX, 1>);
    set((const void*)k_zpass_green<TX, 2>);
  };
  set_tx(std::integral_constant<int, 4>{});
  set_tx(std::integral_constant<int, 8>{});
  set_tx(std::integral_constant<int, 16>{});
  return e;
}

}  // namespace cbs
