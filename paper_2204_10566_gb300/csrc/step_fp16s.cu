// Kernel instantiations for storage precision fp16s (see lbm_device.cuh).
#include "lbm_device.cuh"

namespace lbm {
LBM_INSTANTIATE(2)
}  // namespace lbm
