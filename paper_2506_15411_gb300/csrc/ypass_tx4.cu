// ypass_tx4.cu -- the y-pass kernels of 4-column tiles (yz_kernels.cuh), compiled on their own.
#include "yz_kernels.cuh"

namespace cbs {
CBS_YZ_FUNCS(, 4)
}  // namespace cbs
