// ypass_tx8.cu -- the y-pass kernels of 8-column tiles (yz_kernels.cuh), compiled on their own.
#include "yz_kernels.cuh"

namespace cbs {
CBS_YZ_FUNCS(, 8)
}  // namespace cbs
