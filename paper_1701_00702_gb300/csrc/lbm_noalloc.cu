// Allocation-free diagnostics of caller-owned field arrays.
//
// Some callers cannot allocate device memory: code whose device memory all
// belongs to another allocator (a framework's memory pool, or a serving loop
// that has handed out a fixed HBM budget), and latency-critical paths where
// cudaMalloc/cudaFree would synchronise the device.  lbm_diag_fields_noalloc
// serves them: it reduces fields the caller already holds, and its only
// scratch (one row of four FP64 partial sums per thread block) lives in the
// file-scope array below, which every GPU that loads this library holds until
// the process exits.
#include <cmath>
#include <cstdint>
#include <mutex>

#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 32;
constexpr long long kChunk = (long long)kThreads * kPerThread;     // nodes per block
constexpr int kMaxBlocks = LBM_DIAG_NOALLOC_MAX_NODES / (int)kChunk;  // 8192 blocks
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_partials[kMaxBlocks * 4];

struct Consts {
    double phi, rho_l, rho_m, c_pm, k_f, k_s, k_m;   // k_f liquid, k_s solid PCM conductivity (Eq. 9)
    double nu_scale;   // L / (k_e dT) / ny, or NaN when x = 0 is not a wall
    int nx, ny, left_wall;
};

template <typename R>
__global__ void __launch_bounds__(kThreads) partial_sums(const R* __restrict__ Tf, const R* __restrict__ Ts,
                                                         const R* __restrict__ fl, const R* __restrict__ rho,
                                                         const R* __restrict__ H, const Consts C,
                                                         double* __restrict__ part) {
    const long long n = (long long)C.nx * C.ny;
    const long long begin = (long long)blockIdx.x * kChunk;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < kPerThread; ++j) {
        const long long k = begin + (long long)j * kThreads + threadIdx.x;
        if (k >= n) break;
        v[0] += (double)fl[k];
        v[1] += C.phi * C.rho_l * (double)H[k] + (1.0 - C.phi) * C.rho_m * C.c_pm * (double)Ts[k];
        v[2] += (double)rho[k];
        if (C.left_wall && k % C.nx == 0) {
            const double gf = 0.5 * (3.0 * (double)Tf[k] - 4.0 * (double)Tf[k + 1] + (double)Tf[k + 2]);
            const double gm = 0.5 * (3.0 * (double)Ts[k] - 4.0 * (double)Ts[k + 1] + (double)Ts[k + 2]);
            const double kw = C.k_s == C.k_f ? C.k_f : (double)fl[k] * C.k_f + (1.0 - (double)fl[k]) * C.k_s;
            v[3] += C.phi * kw * gf + (1.0 - C.phi) * C.k_m * gm;
        }
    }
    __shared__ double red[4][kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 0; i < 4; ++i) {
        double a = v[i];
        for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
        if (lane == 0) red[i][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double a = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) a += red[threadIdx.x][w];
        part[(long long)blockIdx.x * 4 + threadIdx.x] = a;   // every block writes its own row
    }
}

__global__ void __launch_bounds__(kThreads) finish(const double* __restrict__ part, int nblocks, const Consts C,
                                                   double* __restrict__ out) {
    __shared__ double red[4][kThreads];
    const int t = threadIdx.x;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = t; b < nblocks; b += kThreads)
        for (int i = 0; i < 4; ++i) a[i] += part[(long long)b * 4 + i];
    for (int i = 0; i < 4; ++i) red[i][t] = a[i];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (t < w)
            for (int i = 0; i < 4; ++i) red[i][t] += red[i][t + w];
        __syncthreads();
    }
    if (t == 0) {
        out[0] = red[0][0] / ((double)C.nx * C.ny);
        out[1] = C.left_wall ? C.nu_scale * red[3][0] : nan("");
        out[2] = red[1][0];
        out[3] = red[2][0];
    }
}

std::mutex g_setup_mutex;

// The device address of g_partials belongs to the module as loaded in one
// CUDA context.  It is looked up once per device and context: a context
// created after cudaDeviceReset may load the module elsewhere, so each
// cached address carries the unique ID of the context it was taken in.
struct Slot {
    double* addr = nullptr;
    unsigned long long ctx_id = 0;
};
Slot g_slots[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Unique ID of the current context (driver entry points, looked up once).
int current_context_id(unsigned long long* id) {
    if (!g_ctx_get_current || !g_ctx_get_id) {
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        void* f1 = nullptr;
        void* f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            cudaGetLastError();
            return LBM_ERR_CUDA;
        }
        g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx || g_ctx_get_id(ctx, id) != CUDA_SUCCESS)
        return LBM_ERR_CUDA;
    return LBM_OK;
}

// Device address of g_partials on the current device: looked up (with that
// device current) on the first call in each context, then cached.
int partials_on_current_device(double** out) {
    int dev = -1;
    // cudaSetDevice makes the device's primary context current on this thread
    // (creating it if needed) without allocating anything
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices || cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long id = 0;
    const int rc = current_context_id(&id);
    if (rc != LBM_OK) return rc;
    Slot& slot = g_slots[dev];
    if (!slot.addr || slot.ctx_id != id) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) {
            cudaGetLastError();
            return LBM_ERR_CUDA;
        }
        slot.addr = static_cast<double*>(p);
        slot.ctx_id = id;
    }
    *out = slot.addr;
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_diag_fields_noalloc(const lbm_params* p, const void* T_f, const void* T_s, const void* f_l,
                                       const void* rho, const void* H_f, double* out, void* cuda_stream) {
    if (!p || !T_f || !T_s || !f_l || !rho || !H_f || !out) return LBM_ERR_ARG;
    lbm_derived d;
    const int rc = lbm_derive(p, &d);
    if (rc != LBM_OK) return rc;
    const long long n = (long long)p->nx * p->ny;
    if (n > LBM_DIAG_NOALLOC_MAX_NODES) return LBM_ERR_TOO_LARGE;
    double* part = nullptr;
    const int src = partials_on_current_device(&part);
    if (src != LBM_OK) return src;

    Consts C;
    C.phi = p->porosity;
    C.rho_l = 1.0;
    C.rho_m = d.rho_m;
    C.c_pm = 1.0;
    C.k_f = p->k_f;
    C.k_s = d.k_s;
    C.k_m = d.k_m;
    C.nx = p->nx;
    C.ny = p->ny;
    C.left_wall = (!p->periodic_x && p->nx >= 3) ? 1 : 0;
    const double k_e = p->porosity * p->k_f + (1.0 - p->porosity) * d.k_m;
    C.nu_scale = p->L_char / (k_e * (p->T_hot - p->T_cold)) / p->ny;
    const int nblocks = (int)((n + kChunk - 1) / kChunk);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (p->precision == LBM_F64)
        partial_sums<double><<<nblocks, kThreads, 0, s>>>(
            static_cast<const double*>(T_f), static_cast<const double*>(T_s), static_cast<const double*>(f_l),
            static_cast<const double*>(rho), static_cast<const double*>(H_f), C, part);
    else
        partial_sums<float><<<nblocks, kThreads, 0, s>>>(
            static_cast<const float*>(T_f), static_cast<const float*>(T_s), static_cast<const float*>(f_l),
            static_cast<const float*>(rho), static_cast<const float*>(H_f), C, part);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    finish<<<1, kThreads, 0, s>>>(part, nblocks, C, out);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    return LBM_OK;
}
