// FP32 storage (float-float PCM rest population): fused step, fields,
// diagnostics and init kernels.
#include "lbm_launch.cuh"

namespace lbmk {
LBMK_INSTANTIATE(MODE_F32)
LBMK_INSTANTIATE_CONVERT(MODE_F32)
}  // namespace lbmk
