// zpass_tx4.cu -- the z-pass kernels of 4-column tiles (yz_kernels.cuh), compiled on their own.
#include "yz_kernels.cuh"

namespace cbs {
CBS_Z_FUNCS(, 4)
}  // namespace cbs
