// FP32 storage: instantiation of the fused step, fields, diagnostics and init kernels.
#include "lbm_launch.cuh"

namespace lbmk {
LBMK_INSTANTIATE(float)
}  // namespace lbmk
