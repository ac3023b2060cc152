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

template <int TX, bool INV>
__global__ void __launch_bounds__(256) k_ypass(const __grid_constant__ CUtensorMap tm, const IterArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* tile = reinterpret_cast<float2*>(smem_raw);   // [nyr][TX]
  float2* scr = tile + a.nyr * TX;                       // [ny][TX]
  float2* tw = scr + a.ny * TX;                          // twiddles of the y axis
  uint64_t& bar = *reinterpret_cast<uint64_t*>(tw + a.twby / sizeof(float2));
  int& fail = *reinterpret_cast<int*>(&bar + 1);
  const int x0 = blockIdx.x * TX, z = blockIdx.y, c = blockIdx.z;
  const int B = a.yb, nbox = a.nyr / B;
  if (!block_setup(tile, &bar, &fail, a.err)) return;
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar, (uint32_t)(nbox * B * TX * sizeof(float2)) + a.twby);
    bulk_load(tw, a.twy, a.twby, &bar);
    for (int b = 0; b < nbox; ++b) tma_load_4d(tile + b * B * TX, &tm, x0, b * B, z, c, &bar);
  }
  if (!block_wait(&bar, &fail, a.err)) return;
  fft_cols<INV, TX>(tile, scr, a.ay, tw, threadIdx.x, blockDim.x);
  fence_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int b = 0; b < nbox; ++b) tma_store_4d(&tm, x0, b * B, z, c, tile + b * B * TX);
    bulk_commit();
    bulk_wait_all();
  }
}

template <int TX>
__global__ void __launch_bounds__(256) k_zpass_green(const __grid_constant__ CUtensorMap tm, const IterArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int nzr = a.nzr, n = a.nz;
  float2* tile = reinterpret_cast<float2*>(smem_raw);   // [3][nzr][TX]
  float2* scr = tile + 3 * nzr * TX;                     // [nz][TX]
  float2* tw = scr + n * TX;                             // twiddles of the z axis
  uint64_t& bar = *reinterpret_cast<uint64_t*>(tw + a.twbz / sizeof(float2));
  int& fail = *reinterpret_cast<int*>(&bar + 1);
  const int x0 = blockIdx.x * TX, y = blockIdx.y;
  const int B = a.zb, nbox = nzr / B;
  if (!block_setup(tile, &bar, &fail, a.err)) return;
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar, (uint32_t)(3 * nbox * B * TX * sizeof(float2)) + a.twbz);
    bulk_load(tw, a.twz, a.twbz, &bar);
    for (int c = 0; c < 3; ++c)
      for (int b = 0; b < nbox; ++b) tma_load_4d(tile + (c * nzr + b * B) * TX, &tm, x0, y, b * B, c, &bar);
  }
  if (!block_wait(&bar, &fail, a.err)) return;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int c = 0; c < 3; ++c) fft_cols<false, TX>(tile + c * nzr * TX, scr, a.az, tw, tid, nth);

  const float two_pi = 6.283185307179586f;
  const float py = two_pi / (float)a.ny * (float)fft_freq(y, a.ny);
  const float qy = (2 * y == a.ny) ? 0.f : py;
  for (int k = tid; k < n * TX; k += nth) {
    const int col = k % TX, i = k / TX;
    const int x = x0 + col;
    const float px = two_pi / (float)a.nx * (float)fft_freq(x, a.nx);
    const float qx = (2 * x == a.nx) ? 0.f : px;
    const float pz = two_pi / (float)n * (float)fft_freq(i, n);
    const float qz = (2 * i == n) ? 0.f : pz;
    float2* e = tile + i * TX + col;
    float2 X0 = e[0], X1 = e[nzr * TX], X2 = e[2 * nzr * TX];
    green(px, py, pz, qx, qy, qz, a.kt2, a.invN, X0, X1, X2);
    e[0] = X0;
    e[nzr * TX] = X1;
    e[2 * nzr * TX] = X2;
  }
  __syncthreads();
  for (int c = 0; c < 3; ++c) fft_cols<true, TX>(tile + c * nzr * TX, scr, a.az, tw, tid, nth);
  fence_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < 3; ++c)
      for (int b = 0; b < nbox; ++b)
        tma_store_4d(&tm, x0, y, b * B, c, tile + (c * nzr + b * B) * TX);
    bulk_commit();
    bulk_wait_all();
  }
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

// tile + scratch + twiddles + 16 bytes for the mbarrier and the failure flag
size_t ypass_smem(const IterArgs& a) { return (size_t)(a.nyr + a.ny) * a.tx_y * sizeof(float2) + a.twby + 16; }
size_t zpass_smem(const IterArgs& a) {
  return (size_t)(3 * a.nzr + a.nz) * a.tx_z * sizeof(float2) + a.twbz + 16;
}

cudaError_t launch_ypass(const CUtensorMap& tm, const IterArgs& a, bool inverse, cudaStream_t s) {
  dim3 grid((a.nx + a.tx_y - 1) / a.tx_y, a.nz, 3);
  return with_tx(a.tx_y, [&](auto T) {
    constexpr int TX = decltype(T)::value;
    if (inverse)
      k_ypass<TX, true><<<grid, 256, ypass_smem(a), s>>>(tm, a);
    else
      k_ypass<TX, false><<<grid, 256, ypass_smem(a), s>>>(tm, a);
    return cudaGetLastError();
  });
}

cudaError_t launch_zpass_green(const CUtensorMap& tm, const IterArgs& a, cudaStream_t s) {
  dim3 grid((a.nx + a.tx_z - 1) / a.tx_z, a.ny, 1);
  return with_tx(a.tx_z, [&](auto T) {
    constexpr int TX = decltype(T)::value;
    k_zpass_green<TX><<<grid, 256, zpass_smem(a), s>>>(tm, a);
    return cudaGetLastError();
  });
}

cudaError_t yzpass_set_smem_limit(int bytes) {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  };
  set((const void*)k_ypass<4, false>);
  set((const void*)k_ypass<4, true>);
  set((const void*)k_ypass<8, false>);
  set((const void*)k_ypass<8, true>);
  set((const void*)k_ypass<16, false>);
  set((const void*)k_ypass<16, true>);
  set((const void*)k_zpass_green<4>);
  set((const void*)k_zpass_green<8>);
  set((const void*)k_zpass_green<16>);
  return e;
}

}  // namespace cbs
