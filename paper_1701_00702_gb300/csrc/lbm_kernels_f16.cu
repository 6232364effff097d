// 16-bit storage (FP16 and BF16 populations, FP32 rest populations and
// arithmetic): fused step, fields, diagnostics, init and state conversion.
#include "lbm_launch.cuh"

namespace lbmk {
LBMK_INSTANTIATE(MODE_F16)
LBMK_INSTANTIATE(MODE_BF16)
LBMK_INSTANTIATE_CONVERT(MODE_F16)
LBMK_INSTANTIATE_CONVERT(MODE_BF16)
}  // namespace lbmk
