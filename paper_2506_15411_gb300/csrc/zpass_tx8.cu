// zpass_tx8.cu -- the z-pass kernels of 8-column tiles (yz_kernels.cuh), compiled on their own.
#include "yz_kernels.cuh"

namespace cbs {
CBS_Z_FUNCS(, 8)
}  // namespace cbs
