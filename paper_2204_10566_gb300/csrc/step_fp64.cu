// Kernel instantiations for storage precision fp64 (see lbm_device.cuh).
#include "lbm_device.cuh"

namespace lbm {
LBM_INSTANTIATE(0)
}  // namespace lbm
