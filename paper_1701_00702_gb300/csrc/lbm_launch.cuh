// Kernel launchers shared by the per-mode translation units.  Each unit
// includes this file and instantiates the launchers for its storage modes.
#pragma once

#include "lbm_kernels.cuh"

namespace lbmk {

constexpr int kBlockX = 128;
constexpr int kBlockY = 2;

inline dim3 grid_for(int nx, int ny) {
    return dim3((unsigned)((nx + kBlockX - 1) / kBlockX), (unsigned)((ny + kBlockY - 1) / kBlockY), 1u);
}

inline int diag_blocks(int nx, int ny) {
    const dim3 g = grid_for(nx, ny);
    return (int)(g.x * g.y);
}

// Uniform initial state: one value per logical population (9 flow, Q PCM, Q
// metal, in the order of Eq. 11), the low part of the PCM rest population
// (MODE_F32), and zero history.
struct InitVals {
    double f[9], g[9], h[9], g0_lo;
};

template <int M, int QT, bool FLOW>
__global__ void init_kernel(const __grid_constant__ StepParams<typename ModeTraits<M>::R> P,
                            const __grid_constant__ InitVals V) {
    using R = typename ModeTraits<M>::R;
    using PL = Planes<M, QT, FLOW>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const int o = y * P.pitch + x;
    if constexpr (FLOW)
        for (int q = 0; q < 9; ++q) stb<M>(const_cast<void*>(P.src[q]), o, (R)(V.f[q] * (double)P.fscale));
    if constexpr (kSplit<M>) {
        const float g0 = (float)V.g[0], h0 = (float)V.h[0];
        static_cast<float*>(const_cast<void*>(P.src[PL::bulk]))[o] = g0;
        static_cast<float*>(const_cast<void*>(P.src[PL::bulk + 1]))[o] = h0;
        for (int q = 1; q < QT; ++q) {
            stb<M>(const_cast<void*>(P.src[PL::pcm(q)]), o, (float)V.g[q] - P.w_move[q] * pcm_ref(P, g0));
            stb<M>(const_cast<void*>(P.src[PL::met(q)]), o, (float)V.h[q] - P.w_move[q] * P.kappa_m * h0);
        }
    } else {
        for (int q = 1; q < QT; ++q) {
            stb<M>(const_cast<void*>(P.src[PL::pcm(q)]), o, (R)V.g[q]);
            stb<M>(const_cast<void*>(P.src[PL::met(q)]), o, (R)V.h[q]);
        }
        stb<M>(const_cast<void*>(P.src[PL::pcm(0)]), o, (R)V.g[0]);
        stb<M>(const_cast<void*>(P.src[PL::met(0)]), o, (R)V.h[0]);
        if constexpr (kComp<M>) stb<M>(const_cast<void*>(P.src[PL::lo]), o, (R)V.g0_lo);
    }
    P.dT[o] = R(0);
}

// Dense float/double copy of the state, [q][ny][nx] per lattice, for the
// 16-bit modes (state I/O converts through it).  to_dense = 1 reads the
// current copy into dense arrays, 0 writes dense arrays into the copy.
struct DenseState {
    float* f;    // 9 planes (deviations f_i - w_i), may be null
    float* g;    // Q planes
    float* h;    // Q planes
};

template <int M, int QT, bool FLOW>
__global__ void convert_state(const __grid_constant__ StepParams<float> P, const __grid_constant__ DenseState D,
                              int to_dense) {
    using PL = Planes<M, QT, FLOW>;
    using B = typename ModeTraits<M>::B;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const int o = y * P.pitch + x;
    const long long k = (long long)y * P.nx + x, dpl = (long long)P.nx * P.ny;
    auto bulk = [&](int plane) { return static_cast<B*>(const_cast<void*>(P.src[plane])); };
    float* wg = static_cast<float*>(const_cast<void*>(P.src[PL::bulk]));
    float* wh = static_cast<float*>(const_cast<void*>(P.src[PL::bulk + 1]));
    if (to_dense) {
        if (FLOW && D.f)
            for (int q = 0; q < 9; ++q) D.f[q * dpl + k] = to_f(bulk(q)[o]) * P.finv;
        if (D.g) {
            const float rg = pcm_ref(P, wg[o]);
            D.g[k] = wg[o];
            for (int q = 1; q < QT; ++q) D.g[q * dpl + k] = to_f(bulk(PL::pcm(q))[o]) + P.w_move[q] * rg;
        }
        if (D.h) {
            const float rm = P.kappa_m * wh[o];
            D.h[k] = wh[o];
            for (int q = 1; q < QT; ++q) D.h[q * dpl + k] = to_f(bulk(PL::met(q))[o]) + P.w_move[q] * rm;
        }
    } else {
        if (FLOW && D.f)
            for (int q = 0; q < 9; ++q) bulk(q)[o] = from_f<B>(D.f[q * dpl + k] * P.fscale);
        if (D.g) {
            const float rg = pcm_ref(P, D.g[k]);
            wg[o] = D.g[k];
            for (int q = 1; q < QT; ++q) bulk(PL::pcm(q))[o] = from_f<B>(D.g[q * dpl + k] - P.w_move[q] * rg);
        }
        if (D.h) {
            const float rm = P.kappa_m * D.h[k];
            wh[o] = D.h[k];
            for (int q = 1; q < QT; ++q) bulk(PL::met(q))[o] = from_f<B>(D.h[q * dpl + k] - P.w_move[q] * rm);
        }
    }
}

template <int M, typename Fn>
inline cudaError_t dispatch(int qt, int flow, Fn&& fn) {
    if (qt == 5) return flow ? fn.template operator()<M, 5, true>() : fn.template operator()<M, 5, false>();
    return flow ? fn.template operator()<M, 9, true>() : fn.template operator()<M, 9, false>();
}

// The step kernels also take PH (the Eq. 9 per-node rates compiled in or not).
template <int M, typename Fn>
inline cudaError_t dispatch_step(int qt, int flow, int ph, Fn&& fn) {
    return dispatch<M>(qt, flow, [&]<int MM, int Q, bool F>() {
        return ph ? fn.template operator()<MM, Q, F, true>() : fn.template operator()<MM, Q, F, false>();
    });
}

template <int M>
cudaError_t launch_step(const StepParams<typename ModeTraits<M>::R>& P, int qt, int flow, cudaStream_t s) {
    const dim3 g = grid_for(P.nx, P.ny), b(kBlockX, kBlockY);
    return dispatch_step<M>(qt, flow, P.phase_k, [&]<int MM, int Q, bool F, bool PH>() {
        fused_step<MM, Q, F, PH><<<g, b, 0, s>>>(P);
        return cudaGetLastError();
    });
}

template <int M>
cudaError_t launch_fields(const StepParams<typename ModeTraits<M>::R>& P,
                          const FieldOut<typename ModeTraits<M>::R>& o, int qt, int flow, cudaStream_t s) {
    const dim3 g = grid_for(P.nx, P.ny), b(kBlockX, kBlockY);
    return dispatch<M>(qt, flow, [&]<int MM, int Q, bool F>() {
        fields_kernel<MM, Q, F><<<g, b, 0, s>>>(P, o);
        return cudaGetLastError();
    });
}

template <int M>
cudaError_t launch_diag(const StepParams<typename ModeTraits<M>::R>& P, const DiagConst& C, double* scratch,
                        double* out, int qt, int flow, cudaStream_t s) {
    const dim3 g = grid_for(P.nx, P.ny), b(kBlockX, kBlockY);
    cudaError_t e = dispatch<M>(qt, flow, [&]<int MM, int Q, bool F>() {
        diag_partial<MM, Q, F><<<g, b, 0, s>>>(P, C, scratch);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    diag_finalize<<<1, 256, 0, s>>>(scratch, (int)(g.x * g.y), out);
    return cudaGetLastError();
}

template <int M>
cudaError_t launch_init(const StepParams<typename ModeTraits<M>::R>& P, const InitVals& V, int qt, int flow,
                        cudaStream_t s) {
    const dim3 g = grid_for(P.nx, P.ny), b(kBlockX, kBlockY);
    return dispatch<M>(qt, flow, [&]<int MM, int Q, bool F>() {
        init_kernel<MM, Q, F><<<g, b, 0, s>>>(P, V);
        return cudaGetLastError();
    });
}

template <int M>
cudaError_t launch_convert(const StepParams<float>& P, const DenseState& D, int to_dense, int qt, int flow,
                           cudaStream_t s) {
    const dim3 g = grid_for(P.nx, P.ny), b(kBlockX, kBlockY);
    return dispatch<M>(qt, flow, [&]<int MM, int Q, bool F>() {
        convert_state<MM, Q, F><<<g, b, 0, s>>>(P, D, to_dense);
        return cudaGetLastError();
    });
}

// ph: some run of the batch uses the Eq. 9 per-node rates.
template <int M>
cudaError_t launch_batch(const StepParams<typename ModeTraits<M>::R>* runs, const Tile* tiles, int ntiles,
                         int chunk, int grid, int parity, int qt, int flow, int ph, cudaStream_t s) {
    return dispatch_step<M>(qt, flow, ph, [&]<int MM, int Q, bool F, bool PH>() {
        batch_step<MM, Q, F, PH><<<grid, 256, 0, s>>>(runs, tiles, ntiles, chunk, parity);
        return cudaGetLastError();
    });
}

// The single-run kernel as a function pointer, for kernel nodes built
// directly into a graph (one chain of steps per run).
template <int M>
const void* step_kernel(int qt, int flow, int ph) {
    const void* fn = nullptr;
    dispatch_step<M>(qt, flow, ph, [&]<int MM, int Q, bool F, bool PH>() {
        fn = (const void*)fused_step<MM, Q, F, PH>;
        return cudaSuccess;
    });
    return fn;
}

template <int M>
int batch_blocks_per_sm(int qt, int flow, int ph) {
    int n = 0;
    dispatch_step<M>(qt, flow, ph, [&]<int MM, int Q, bool F, bool PH>() {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step<MM, Q, F, PH>, 256, 0);
    });
    return n;
}

#define LBMK_INSTANTIATE(M)                                                                                   \
    template cudaError_t launch_step<M>(const StepParams<ModeTraits<M>::R>&, int, int, cudaStream_t);        \
    template cudaError_t launch_fields<M>(const StepParams<ModeTraits<M>::R>&, const FieldOut<ModeTraits<M>::R>&, \
                                          int, int, cudaStream_t);                                            \
    template cudaError_t launch_diag<M>(const StepParams<ModeTraits<M>::R>&, const DiagConst&, double*, double*, \
                                        int, int, cudaStream_t);                                              \
    template cudaError_t launch_init<M>(const StepParams<ModeTraits<M>::R>&, const InitVals&, int, int, cudaStream_t); \
    template cudaError_t launch_batch<M>(const StepParams<ModeTraits<M>::R>*, const Tile*, int, int, int, int, int, \
                                         int, int, cudaStream_t);                                               \
    template int batch_blocks_per_sm<M>(int, int, int);                                                   \
    template const void* step_kernel<M>(int, int, int);

#define LBMK_INSTANTIATE_CONVERT(M) \
    template cudaError_t launch_convert<M>(const StepParams<float>&, const DenseState&, int, int, int, cudaStream_t);

}  // namespace lbmk
