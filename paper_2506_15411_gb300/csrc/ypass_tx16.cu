// ypass_tx16.cu -- the y-pass kernels of 16-column tiles (yz_kernels.cuh), compiled on their own.
#include "yz_kernels.cuh"

namespace cbs {
CBS_YZ_FUNCS(, 16)
}  // namespace cbs
