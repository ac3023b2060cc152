// cbs_internal.h -- structures shared by the host library and the CUDA kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstddef>

#include "fft_ip.cuh"

namespace cbs {

constexpr int kBoxRows = 64;   // at most this many rows (y or z) per tensor-copy box

// Source term in the scaled units of the kernels (all k^2 quantities times pitch^2).
struct SourceArgs {
  int kind;               // 0 plane wave, 1 point, 2 user array
  float2 amp[3];          // plane wave: pol * (-2 i k_b pitch); point: pol * pitch^2
  int zp;                 // plane-wave sheet
  int px, py, pz;         // point-source voxel
  const float2* amp_dev;  // point source with amplitudes on the device (adjoint), or null
  const float2* user;     // user S [3][N]
  float user_scale;       // pitch^2
};

// Requests that share one launch: a plan's arrays (E, W, V) hold `seats` requests of the same
// grid side by side, and a launch iterates up to kMaxMembers of them, each with its own source
// and splitting (an array of Member in device memory, written before the launch).  A launch's
// grid is nmem times the per-request persistent grid; block b works for member b / grid, as
// block b mod grid of that request's own persistent grid, so every request's tiles, and the
// order of its residual sums, are the same in any launch.
constexpr int kMaxMembers = 8;

struct Member {
  SourceArgs src;
  float inv_eps;          // 1 / epsilon (scaled)
  float2 kt2;             // k0^2 + i epsilon (scaled)
  int seat;               // slice of the plan's arrays: E, W at + seat * 3 Nw; V at + seat * Nw
};

// Everything one CBS iteration needs (kernel parameters, by value).
struct IterArgs {
  int nx, ny, nz;
  size_t N;               // nx * ny * nz (fields E, V, sources: dense rows)
  int nxp;                // row pitch of the workspace W (multiple of 16 complex values)
  int yblk, nyb;          // y-blocked layout: blocks of yblk y rows (yblk divides ny), nyb blocks
  size_t Nw;              // nxp * ny * nz: component stride of W, E
  int yb, zb;             // rows per tensor-copy box along y and z
  int nyr, nzr;           // ny, nz rounded up to whole boxes (shared-memory rows of a tile)
  AxisIP ax, ay, az;      // in-place FFT plans (fft_ip.cuh)
  const float2* twx;      // per-stage twiddle tables; each 128-byte aligned, padded to n entries
  const float2* twy;
  const float2* twz;
  int twbx, twby, twbz;   // bytes copied per table: n * 8 rounded up to a multiple of 16
  const float2* pqx;      // wave numbers (p, q) of each position of an axis' spectrum,
  const float2* pqy;      // padded with zeros to a multiple of 16 entries
  const float2* pqz;
  int pqbz;               // bytes of the z table the z pass copies (multiple of 16)
  float2* E;              // fields being iterated, [seats][3][nyb][nz][yblk][nxp] (plan-owned)
  float2* W;              // workspace, same layout
  const float2* V;        // potential [seats][nyb][nz][yblk][nxp], scaled
  int seats;              // requests the arrays hold
  int nmem;               // members of this launch (1 .. kMaxMembers)
  const Member* mem;      // their sources, splittings and seats (device memory)
  float invN;             // 1 / N, folded into the k-space multiply
  double* partials;       // residual partial sums, [seat][grid_x]
  unsigned* counter;      // last-block-done counters, [seat] (left at 0)
  double* hist;           // hist[seat * hist_cap + slot] = sum |delta|^2 of this iteration
  int hist_cap;
  int slot;
  int* err;               // device error flag (a tensor-copy wait that timed out)
  // launch shapes
  int rpb;                // rows per tile, x passes
  int nset_x, nset_xf;    // buffer sets of the x passes (inverse + forward; first forward)
  int tx_y, tx_z;         // x-columns per tile, y and z passes
  int nbuf_y, nbuf_z;     // tile buffers of the pipelined y and z passes (2 to 4)
  int occ_y, occ_z;       // blocks per SM of the y and z kernels (2: radices <= 11, 64 registers)
  int maxr_x, maxr_z;     // largest radix of the x and z axes (selects the kernel build)
  int xgroups, zgroups;   // warp groups of the fused x and the z blocks (1 or 2)
  int grid_x, grid_xf, grid_y, grid_z;   // persistent grid sizes of one request (x inverse,
                                         // x forward, y, z); a launch has nmem times as many
};

// Block b of a launch: member b / G, block b mod G of that member's grid of G blocks.
struct MemberBlock {
  int j, b;
};
CBS_HD MemberBlock member_block(int block, int G) {
  const int j = block / G;
  return MemberBlock{j, block - j * G};
}

// The plan's arrays (W, the iterate E, V) store row (y, z) of a component at
//     ((y / yblk) * nz + z) * yblk + y mod yblk
// -- blocks of yblk consecutive y rows, z inside a block: a z column then visits rows yblk
// rows apart (instead of ny), and a y column runs in nyb stretches of yblk rows.  Long
// z strides of the plain [z][y] order slowed the z pass by half on a 640 x 640 plane.
CBS_HD size_t wrow(int y, int z, int nz, int yblk) {
  const int yb = y / yblk;
  return ((size_t)yb * nz + z) * yblk + (y - yb * yblk);
}

// Launchers (one per pass of an iteration); each returns the launch error.
cudaError_t launch_xpass_fwd(const IterArgs& a, cudaStream_t s);   // W = FFTx(V E + S)
cudaError_t launch_ypass(const CUtensorMap& tm, const IterArgs& a, bool inverse, cudaStream_t s);
cudaError_t launch_zpass_green(const CUtensorMap& tm, const IterArgs& a, cudaStream_t s);  // FFTz, G, IFFTz
cudaError_t launch_xpass_inv_fwd(const IterArgs& a, cudaStream_t s);  // IFFTx, update, residual, next FFTx

// Shared-memory bytes and threads of each pass for the plan's shapes.
size_t xpass_smem(const IterArgs& a);
int xpass_tiles(const IterArgs& a);
cudaError_t yz_grid_sizes(IterArgs& a, int sms);   // sets grid_y, grid_z
cudaError_t x_grid_size(IterArgs& a, int sms);     // sets grid_x, grid_xf

// Set-up and gradient kernels (misc.cu).
cudaError_t launch_eps_minmax(const float* eps, size_t N, float* part_min, float* part_max,
                              int* part_bad, int blocks, cudaStream_t s);
cudaError_t launch_k2_maxdev(const float* eps, int nx, int ny, int nz, const double* sx,
                             const double* sy, const double* sz, int corner_max, double kv2, double k0sq,
                             double* part, int blocks, cudaStream_t s);
cudaError_t launch_build_v(const float* eps, int nx, int ny, int nz, int nxp, int yblk, const double* sx,
                           const double* sy, const double* sz, int corner_max, double kv2, double k0sq,
                           double eps_shift, float2* V, cudaStream_t s);
// A field between the caller's dense layout [3][nz][ny][nx] and the plan's y-blocked one
// (to_dense: plan -> dense); the row padding of the plan's copy is not written.
cudaError_t launch_field_layout(const float2* src, float2* dst, bool to_dense, int nx, int ny, int nz, int nxp,
                                int yblk, cudaStream_t s);
cudaError_t launch_adjoint_amp(const float2* E, size_t N, int nx, int ny, int x, int y, int z,
                               float scale, float2* amp, cudaStream_t s);
cudaError_t launch_gradient(const float2* E, const float2* Ea, size_t N, float coef, float* g,
                            cudaStream_t s);
cudaError_t launch_objective(const float2* E, size_t N, int nx, int ny, int x, int y, int z,
                             double* out, cudaStream_t s);

// Bounded-wait self-test (misc.cu): *err = 1 (tensor-copy wait timed out) after `limit` polls.
cudaError_t launch_wait_selftest(int* err, long long limit, cudaStream_t s);

// Inverse-design kernels on the thickness map (design.cu).
cudaError_t launch_mirror(const float* in, float* out, int nx, int ny, cudaStream_t s);
cudaError_t launch_filter(const float* in, float* out, int nx, int ny, const float* w, int R, int axis,
                          cudaStream_t s);
cudaError_t launch_height_to_eps(const float* heff, float* eps, int nx, int ny, int nz, int z_base, float inv_pitch,
                                 float eb, float de, int sms, cudaStream_t s);
cudaError_t launch_surface_grad(const float* g, const float* heff, float* out, int nx, int ny, int nz, int z_base,
                                float inv_pitch, float slope, cudaStream_t s);
cudaError_t launch_adam(float* h, const float* gh, float* m, float* v, int nx, int ny, double pitch_um,
                        double r2max, float alpha, float b1, float b2, float c1, float c2, float aeps, float hmax,
                        cudaStream_t s);

}  // namespace cbs
