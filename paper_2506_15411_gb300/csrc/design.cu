// design.cu -- kernels of one inverse-design step on the lens thickness map h(x, y)
// (Section 3 and Fig. 2(a) of arXiv 2506.15411):
//   h_eff = G_sigma[M h]            mirror average M, separable Gaussian G_sigma (zero outside)
//   eps_r = eps_bg + f (eps_lens - eps_bg),  f = clamp(h_eff / pitch - (z - z_base), 0, 1)
//   dL/dh_eff = (eps_lens - eps_bg) / pitch * dL/d eps_r at the voxel z_base + floor(h_eff / pitch)
//   dL/dh = M G_sigma [dL/dh_eff]   (both operators are symmetric)
//   Adam ascent on L, then 0 <= h <= h_max inside the aperture and h = 0 outside it.
// Maps are float32 [ny][nx] in micrometres; the volume is float32 [nz][ny][nx].  All of it
// is a few light passes next to the CBS solves, so the kernels are plain one-thread-per-
// element loops with coalesced x.
#include <algorithm>

#include "cbs_internal.h"

namespace cbs {
namespace {

// ((h(x,y) + h(X,y)) + (h(x,Y) + h(X,Y))) / 4 with X = nx-1-x, Y = ny-1-y: the pairwise order
// makes the result exactly symmetric.
__global__ void k_mirror(const float* __restrict__ in, float* __restrict__ out, int nx, int ny) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= nx) return;
  const int X = nx - 1 - x, Y = ny - 1 - y;
  const float a = in[(size_t)y * nx + x] + in[(size_t)y * nx + X];
  const float b = in[(size_t)Y * nx + x] + in[(size_t)Y * nx + X];
  out[(size_t)y * nx + x] = 0.25f * (a + b);
}

// out[i] = w_0 in[i] + sum_{k=1..R} w_k (in[i + k] + in[i - k]) along x (axis 0) or y
// (axis 1), zero outside the map; w holds w_0 .. w_R.  Summing the mirror pairs first keeps a
// mirror-symmetric input exactly symmetric.
__global__ void k_filter(const float* __restrict__ in, float* __restrict__ out, int nx, int ny,
                         const float* __restrict__ w, int R, int axis) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= nx) return;
  const size_t p = (size_t)y * nx + x;
  const int i = axis == 0 ? x : y, n = axis == 0 ? nx : ny;
  const size_t st = axis == 0 ? 1 : (size_t)nx;
  float acc = __ldg(&w[0]) * in[p];
  for (int k = 1; k <= R; ++k) {
    const float a = (i + k < n) ? in[p + k * st] : 0.f;
    const float b = (i - k >= 0) ? in[p - k * st] : 0.f;
    acc = fmaf(__ldg(&w[k]), a + b, acc);
  }
  out[p] = acc;
}

__global__ void k_height_to_eps(const float* __restrict__ heff, float* __restrict__ eps, int nx, int ny, int nz,
                                int z_base, float inv_pitch, float eb, float de) {
  const size_t nxy = (size_t)nx * ny, N = nxy * nz;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const int z = (int)(i / nxy);
    const int k = z - z_base;
    float f = 0.f;
    if (k >= 0) f = fminf(fmaxf(heff[i - (size_t)z * nxy] * inv_pitch - (float)k, 0.f), 1.f);
    eps[i] = fmaf(f, de, eb);
  }
}

__global__ void k_surface_grad(const float* __restrict__ g, const float* __restrict__ heff, float* __restrict__ out,
                               int nx, int ny, int nz, int z_base, float inv_pitch, float slope) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= nx) return;
  const size_t p = (size_t)y * nx + x;
  const float u = heff[p] * inv_pitch;
  float v = 0.f;
  if (u >= 0.f && u < (float)(nz - z_base)) {   // also false for NaN; keeps the cast in range
    const int z = z_base + (int)floorf(u);
    v = slope * g[(size_t)z * nx * ny + p];
  }
  out[p] = v;
}

// Adam (Kingma & Ba, Algorithm 1) on the loss -L, bias corrections c1 = 1/(1 - beta1^t),
// c2 = 1/(1 - beta2^t); the aperture test r^2 <= r2max is taken in FP64 without contraction.
__global__ void k_adam(float* __restrict__ h, const float* __restrict__ gh, float* __restrict__ m,
                       float* __restrict__ v, int nx, int ny, double pitch_um, double r2max, float alpha,
                       float b1, float b2, float c1, float c2, float aeps, float hmax) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= nx) return;
  const size_t p = (size_t)y * nx + x;
  const double xc = __dmul_rn((double)x - 0.5 * (nx - 1), pitch_um);
  const double yc = __dmul_rn((double)y - 0.5 * (ny - 1), pitch_um);
  if (!(__dadd_rn(__dmul_rn(xc, xc), __dmul_rn(yc, yc)) <= r2max)) {
    h[p] = 0.f;
    return;
  }
  const float g = -gh[p];
  const float mi = b1 * m[p] + (1.f - b1) * g;
  const float vi = b2 * v[p] + (1.f - b2) * g * g;
  m[p] = mi;
  v[p] = vi;
  const float step = alpha * (mi * c1) / (sqrtf(vi * c2) + aeps);
  h[p] = fminf(fmaxf(h[p] - step, 0.f), hmax);
}

dim3 map_grid(int nx, int ny) { return dim3((nx + 127) / 128, ny); }

}  // namespace

cudaError_t launch_mirror(const float* in, float* out, int nx, int ny, cudaStream_t s) {
  k_mirror<<<map_grid(nx, ny), 128, 0, s>>>(in, out, nx, ny);
  return cudaGetLastError();
}

cudaError_t launch_filter(const float* in, float* out, int nx, int ny, const float* w, int R, int axis,
                          cudaStream_t s) {
  k_filter<<<map_grid(nx, ny), 128, 0, s>>>(in, out, nx, ny, w, R, axis);
  return cudaGetLastError();
}

cudaError_t launch_height_to_eps(const float* heff, float* eps, int nx, int ny, int nz, int z_base, float inv_pitch,
                                 float eb, float de, int sms, cudaStream_t s) {
  const size_t N = (size_t)nx * ny * nz;
  const size_t want = (N + 255) / 256;
  const int blocks = (int)std::min<size_t>(want, (size_t)sms * 16);
  k_height_to_eps<<<blocks, 256, 0, s>>>(heff, eps, nx, ny, nz, z_base, inv_pitch, eb, de);
  return cudaGetLastError();
}

cudaError_t launch_surface_grad(const float* g, const float* heff, float* out, int nx, int ny, int nz, int z_base,
                                float inv_pitch, float slope, cudaStream_t s) {
  k_surface_grad<<<map_grid(nx, ny), 128, 0, s>>>(g, heff, out, nx, ny, nz, z_base, inv_pitch, slope);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* h, const float* gh, float* m, float* v, int nx, int ny, double pitch_um,
                        double r2max, float alpha, float b1, float b2, float c1, float c2, float aeps, float hmax,
                        cudaStream_t s) {
  k_adam<<<map_grid(nx, ny), 128, 0, s>>>(h, gh, m, v, nx, ny, pitch_um, r2max, alpha, b1, b2, c1, c2, aeps, hmax);
  return cudaGetLastError();
}

}  // namespace cbs
