// yzpass.cu -- host side of the strided passes (y, and z with the k-space multiply): launch
// shapes, grid sizes and launches.  The kernels are in yz_kernels.cuh and are compiled per
// tile width in ypass_tx*.cu / zpass_tx*.cu.
#include <algorithm>

#include "yz_kernels.cuh"

namespace cbs {

CBS_YZ_FUNCS(extern, 4)
CBS_YZ_FUNCS(extern, 8)
CBS_YZ_FUNCS(extern, 16)
CBS_Z_FUNCS(extern, 4)
CBS_Z_FUNCS(extern, 8)
CBS_Z_FUNCS(extern, 16)

namespace {

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

int ypass_tiles(const IterArgs& a) { return (a.nx + a.tx_y - 1) / a.tx_y * a.nz * 3; }
int zpass_tiles(const IterArgs& a) { return (a.nx + a.tx_z - 1) / a.tx_z * a.ny; }

// Persistent grids: as many blocks as fit on the device at once (capped by the tile count).
cudaError_t yz_grid_sizes(IterArgs& a, int sms) {
  int occ = 0;
  cudaError_t e = with_tx(a.tx_y, [&](auto T) { return y_occupancy<decltype(T)::value>(a, &occ); });
  if (e != cudaSuccess) return e;
  a.grid_y = std::max(1, std::min(ypass_tiles(a), sms * std::max(1, occ)));
  e = with_tx(a.tx_z, [&](auto T) { return z_occupancy<decltype(T)::value>(a, &occ); });
  if (e != cudaSuccess) return e;
  a.grid_z = std::max(1, std::min(zpass_tiles(a), sms * std::max(1, occ)));
  return cudaSuccess;
}

cudaError_t launch_ypass(const CUtensorMap& tm, const IterArgs& a, bool inverse, cudaStream_t s) {
  return with_tx(a.tx_y, [&](auto T) { return y_launch<decltype(T)::value>(tm, a, inverse, s); });
}

cudaError_t launch_zpass_green(const CUtensorMap& tm, const IterArgs& a, cudaStream_t s) {
  return with_tx(a.tx_z, [&](auto T) { return z_launch<decltype(T)::value>(tm, a, s); });
}

cudaError_t yzpass_set_smem_limit(int bytes) {
  cudaError_t e = cudaSuccess;
  for (int tx : {4, 8, 16}) {
    if (e == cudaSuccess) e = with_tx(tx, [&](auto T) { return y_set_smem<decltype(T)::value>(bytes); });
    if (e == cudaSuccess) e = with_tx(tx, [&](auto T) { return z_set_smem<decltype(T)::value>(bytes); });
  }
  return e;
}

}  // namespace cbs
