// Kernel instantiations for storage precision fp32 (see lbm_device.cuh).
#include "lbm_device.cuh"

namespace lbm {
LBM_INSTANTIATE(1)
}  // namespace lbm
