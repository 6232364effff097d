// FP64 storage: instantiation of the fused step, fields, diagnostics and init
// kernels, plus the precision-independent diagnostics finalizer.
#include "lbm_launch.cuh"

namespace lbmk {
LBMK_INSTANTIATE(MODE_F64)
LBMK_INSTANTIATE_CONVERT(MODE_F64)

// Fixed-order sum of the per-block partials: thread t adds blocks t, t+256, ...
// then a shared-memory tree combines the 256 thread sums; out[0..3] =
// sum f_l, sum enthalpy, sum rho, sum left-wall flux.
__global__ void diag_finalize(const double* __restrict__ scratch, int nblocks, double* __restrict__ out) {
    __shared__ double red[4][256];
    const int t = threadIdx.x;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = t; b < nblocks; b += blockDim.x)
        for (int i = 0; i < 4; ++i) a[i] += scratch[(long long)b * 4 + i];
    for (int i = 0; i < 4; ++i) red[i][t] = a[i];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (t < w)
            for (int i = 0; i < 4; ++i) red[i][t] += red[i][t + w];
        __syncthreads();
    }
    if (t < 4) out[t] = red[t][0];
}
}  // namespace lbmk
