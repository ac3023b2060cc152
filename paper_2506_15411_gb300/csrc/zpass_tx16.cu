// zpass_tx16.cu -- the z-pass kernels of 16-column tiles (yz_kernels.cuh), compiled on their own.
#include "yz_kernels.cuh"

namespace cbs {
CBS_Z_FUNCS(, 16)
}  // namespace cbs
