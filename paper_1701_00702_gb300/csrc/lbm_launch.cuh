// Kernel launchers shared by the per-precision translation units.  Each unit
// includes this file and instantiates the launchers for its storage type.
#pragma once

#include "lbm_kernels.cuh"

namespace lbmk {

constexpr int kBlockX = 128;
constexpr int kBlockY = 2;

inline dim3 grid_for(int nx, int ny) {
    return dim3((unsigned)((nx + kBlockX - 1) / kBlockX), (unsigned)((ny + kBlockY - 1) / kBlockY), 1u);
}

template <typename R>
struct InitVals {
    R v[28];   // one value per plane: 9 flow + 9 PCM + 9 metal + low part of g_0
};

template <typename R>
__global__ void init_kernel(R* __restrict__ buf, R* __restrict__ dT, int nplanes, long long plane,
                            int nx, int ny, int pitch, const __grid_constant__ InitVals<R> V) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const long long o = (long long)y * pitch + x;
    for (int p = 0; p < nplanes; ++p) buf[p * plane + o] = V.v[p];
    dT[o] = R(0);
}

template <typename R, int QT, bool FLOW>
inline cudaError_t launch_step_t(const StepParams<R>& P, cudaStream_t s) {
    fused_step<R, QT, FLOW><<<grid_for(P.nx, P.ny), dim3(kBlockX, kBlockY), 0, s>>>(P);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_step(const StepParams<R>& P, int qt, int flow, cudaStream_t s) {
    if (qt == 5) return flow ? launch_step_t<R, 5, true>(P, s) : launch_step_t<R, 5, false>(P, s);
    return flow ? launch_step_t<R, 9, true>(P, s) : launch_step_t<R, 9, false>(P, s);
}

template <typename R>
cudaError_t launch_fields(const StepParams<R>& P, const FieldOut<R>& o, int qt, int flow, cudaStream_t s) {
    const dim3 g = grid_for(P.nx, P.ny), b(kBlockX, kBlockY);
    if (qt == 5) {
        if (flow) fields_kernel<R, 5, true><<<g, b, 0, s>>>(P, o);
        else fields_kernel<R, 5, false><<<g, b, 0, s>>>(P, o);
    } else {
        if (flow) fields_kernel<R, 9, true><<<g, b, 0, s>>>(P, o);
        else fields_kernel<R, 9, false><<<g, b, 0, s>>>(P, o);
    }
    return cudaGetLastError();
}

inline int diag_blocks(int nx, int ny) {
    const dim3 g = grid_for(nx, ny);
    return (int)(g.x * g.y);
}

template <typename R>
cudaError_t launch_diag(const StepParams<R>& P, const DiagConst& C, double* scratch, double* out,
                        int qt, int flow, cudaStream_t s) {
    const dim3 g = grid_for(P.nx, P.ny), b(kBlockX, kBlockY);
    if (qt == 5) {
        if (flow) diag_partial<R, 5, true><<<g, b, 0, s>>>(P, C, scratch);
        else diag_partial<R, 5, false><<<g, b, 0, s>>>(P, C, scratch);
    } else {
        if (flow) diag_partial<R, 9, true><<<g, b, 0, s>>>(P, C, scratch);
        else diag_partial<R, 9, false><<<g, b, 0, s>>>(P, C, scratch);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_finalize<<<1, 256, 0, s>>>(scratch, (int)(g.x * g.y), out);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_init(R* buf, R* dT, int nplanes, long long plane, int nx, int ny, int pitch,
                        const InitVals<R>& V, cudaStream_t s) {
    init_kernel<R><<<grid_for(nx, ny), dim3(kBlockX, kBlockY), 0, s>>>(buf, dT, nplanes, plane, nx, ny, pitch, V);
    return cudaGetLastError();
}

#define LBMK_INSTANTIATE(R)                                                                              \
    template cudaError_t launch_step<R>(const StepParams<R>&, int, int, cudaStream_t);                   \
    template cudaError_t launch_fields<R>(const StepParams<R>&, const FieldOut<R>&, int, int, cudaStream_t); \
    template cudaError_t launch_diag<R>(const StepParams<R>&, const DiagConst&, double*, double*, int, int, \
                                        cudaStream_t);                                                   \
    template cudaError_t launch_init<R>(R*, R*, int, long long, int, int, int, const InitVals<R>&, cudaStream_t);

}  // namespace lbmk
