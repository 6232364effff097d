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
    auto* db = bulk_at<M, QT, FLOW>(const_cast<char*>(P.src), P, x, y);
    if constexpr (FLOW)
        for (int q = 0; q < 9; ++q) stb<M>(db + q * kChunk, (R)(V.f[q] * (double)P.fscale));
    if constexpr (kSplit<M>) {
        float* dw = wide_at<M, QT, FLOW>(const_cast<char*>(P.src), P, x, y);
        const float g0 = (float)V.g[0], h0 = (float)V.h[0];
        dw[0] = g0;
        dw[kChunk] = h0;
        for (int q = 1; q < QT; ++q) {
            stb<M>(db + PL::pcm(q) * kChunk, (float)V.g[q] - P.w_move[q] * pcm_ref(P, g0));
            stb<M>(db + PL::met(q) * kChunk, (float)V.h[q] - P.w_move[q] * P.kappa_m * h0);
        }
    } else {
        for (int q = 0; q < QT; ++q) {
            stb<M>(db + PL::pcm(q) * kChunk, (R)V.g[q]);
            stb<M>(db + PL::met(q) * kChunk, (R)V.h[q]);
        }
        if constexpr (kComp<M>) stb<M>(db + PL::lo * kChunk, (R)V.g0_lo);
    }
    P.dT[y * P.pitch + x] = R(0);
}

// Dense copy of the state, [q][ny][nx] per lattice in the run's arithmetic
// type (state I/O converts through it).  to_dense = 1 reads the current copy
// into the dense arrays, 0 writes the dense arrays into the copy; a null
// array is skipped.  The 16-bit modes decode (encode) the moving thermal
// populations with the reference of their node; FP32 carries the low part
// of the PCM rest population in lo (taken as zero on writing when lo is null
// and g is given).
template <typename R>
struct DenseState {
    R* f;      // 9 planes (deviations f_i - w_i)
    R* g;      // Q planes
    R* h;      // Q planes
    R* lo;     // FP32 only: low part of g_0
};

template <int M, int QT, bool FLOW>
__global__ void convert_state(const __grid_constant__ StepParams<typename ModeTraits<M>::R> P,
                              const __grid_constant__ DenseState<typename ModeTraits<M>::R> D, int to_dense) {
    using R = typename ModeTraits<M>::R;
    using B = typename ModeTraits<M>::B;
    using PL = Planes<M, QT, FLOW>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long k = (long long)y * P.nx + x, dpl = (long long)P.nx * P.ny;
    B* db = bulk_at<M, QT, FLOW>(const_cast<char*>(P.src), P, x, y);
    if (to_dense) {
        if (FLOW && D.f)
            for (int q = 0; q < 9; ++q) D.f[q * dpl + k] = to_f(db[q * kChunk]) * P.finv;
        if constexpr (kSplit<M>) {
            const float* dw = wide_at<M, QT, FLOW>(P.src, P, x, y);
            if (D.g) {
                const float rg = pcm_ref(P, dw[0]);
                D.g[k] = dw[0];
                for (int q = 1; q < QT; ++q) D.g[q * dpl + k] = to_f(db[PL::pcm(q) * kChunk]) + P.w_move[q] * rg;
            }
            if (D.h) {
                const float rm = P.kappa_m * dw[kChunk];
                D.h[k] = dw[kChunk];
                for (int q = 1; q < QT; ++q) D.h[q * dpl + k] = to_f(db[PL::met(q) * kChunk]) + P.w_move[q] * rm;
            }
        } else {
            if (D.g)
                for (int q = 0; q < QT; ++q) D.g[q * dpl + k] = to_f(db[PL::pcm(q) * kChunk]);
            if (D.h)
                for (int q = 0; q < QT; ++q) D.h[q * dpl + k] = to_f(db[PL::met(q) * kChunk]);
            if constexpr (kComp<M>)
                if (D.lo) D.lo[k] = db[PL::lo * kChunk];
        }
    } else {
        if (FLOW && D.f)
            for (int q = 0; q < 9; ++q) db[q * kChunk] = from_f<B>(D.f[q * dpl + k] * P.fscale);
        if constexpr (kSplit<M>) {
            float* dw = wide_at<M, QT, FLOW>(const_cast<char*>(P.src), P, x, y);
            if (D.g) {
                const float rg = pcm_ref(P, D.g[k]);
                dw[0] = D.g[k];
                for (int q = 1; q < QT; ++q) db[PL::pcm(q) * kChunk] = from_f<B>(D.g[q * dpl + k] - P.w_move[q] * rg);
            }
            if (D.h) {
                const float rm = P.kappa_m * D.h[k];
                dw[kChunk] = D.h[k];
                for (int q = 1; q < QT; ++q) db[PL::met(q) * kChunk] = from_f<B>(D.h[q * dpl + k] - P.w_move[q] * rm);
            }
        } else {
            if (D.g)
                for (int q = 0; q < QT; ++q) db[PL::pcm(q) * kChunk] = from_f<B>(D.g[q * dpl + k]);
            if (D.h)
                for (int q = 0; q < QT; ++q) db[PL::met(q) * kChunk] = from_f<B>(D.h[q * dpl + k]);
            if constexpr (kComp<M>)
                if (D.lo || D.g) db[PL::lo * kChunk] = D.lo ? D.lo[k] : R(0);
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

// Block shape of the single-run step kernel by grid size (measured on GB300,
// us per step: 128^2 and 192^2 finish sooner in 64 x 2 blocks, 1.63 and 1.86
// against 1.73 and 2.11 in 128 x 1; from 256^2 up one-row blocks do as well or
// better, 2.37 against 2.47 at 256^2).
inline dim3 step_block(int nx, int ny) {
    return (long long)nx * ny <= 40000 ? dim3(64, 2) : dim3(128, 1);
}

// Step forms: one node per thread (fused_step) or node pairs
// (fused_step_pair, the default configuration only: flow, D2Q5, volumetric
// blend, FP32 arithmetic).  Automatic: node pairs, with the L2 prefetch, for
// the 16-bit forms from 1536 x 1024 nodes up (measured on GB300, us per step:
// FP16 2048^2 62.1 against 72.7, 2048 x 1024 34.1 against 38.1, 1448^2 37.3
// against 39.2; at 1024^2, whose state nearly fits in L2, one node per thread
// is faster, 18.9 against 19.4; in FP32, bound by HBM, one node per thread is
// faster at every size).
enum : int { FORM_AUTO = 0, FORM_SINGLE = 1, FORM_PAIRS = 2, FORM_TWO_STEPS = 3 };
constexpr long long kPairMinNodes = 3ll << 19;

// The rule (host code; lbm_step_form_for reports it): the form a run takes,
// FORM_SINGLE or FORM_PAIRS.  mode: MODE_*.
inline int form_for(int mode, int qt, int flow, int solid_scheme, long long nodes, int form) {
    const bool pairs = mode != MODE_F64 && qt == 5 && flow && !solid_scheme;
    if (form == FORM_PAIRS) return pairs ? FORM_PAIRS : FORM_SINGLE;
    if (form == FORM_SINGLE || form == FORM_TWO_STEPS) return FORM_SINGLE;
    if (pairs && (mode == MODE_F16 || mode == MODE_BF16) && nodes >= kPairMinNodes) return FORM_PAIRS;
    return FORM_SINGLE;
}

// Two time steps per launch (fused_step2) for runs with flow in FP32, FP16
// or BF16 storage: forced by FORM_TWO_STEPS; automatic, for the D2Q5 thermal
// lattices, on grids of up to kTwoStepSmallMaxNodes nodes (the launch floor and
// one dependency chain per step dominate there) and for FP32 on grids of at
// least kTwoStepF32MinNodes (two state copies, 168 bytes per node, exceed the
// 129 MB L2, and two steps per launch move the state through HBM once per two
// steps).  Between the two the state sits in L2 and the step is bound by
// instruction issue, which the redundant ring only adds to (us per step, one
// against two steps per launch; FP32: 256^2 2.40 / 2.02, 320^2 3.01 / 2.74,
// 352^2 3.16 / 3.30, 384^2 3.39 / 4.26, 512^2 4.99 / 5.98, 768^2 11.1 / 12.2,
// 896^2 19.1 / 16.9, 1024^2 26.5 / 21.9, 2048^2 99.7 / 81.2; FP16: 320^2
// 3.14 / 2.91, 352^2 3.20 / 4.25).  Single steps (an odd remainder, batches)
// keep the form above.
constexpr long long kTwoStepSmallMaxNodes = 320 * 320;
constexpr long long kTwoStepF32MinNodes = 3ll << 18;

inline bool two_steps_for(int mode, int qt, int flow, long long nodes, int form) {
    const bool can = mode != MODE_F64 && flow;
    if (form == FORM_TWO_STEPS) return can;
    if (form != FORM_AUTO || !can || qt != 5) return false;
    return nodes <= kTwoStepSmallMaxNodes || (mode == MODE_F32 && nodes >= kTwoStepF32MinNodes);
}

template <int M>
inline int form_of(const StepParams<typename ModeTraits<M>::R>& P, int qt, int flow, int form) {
    return form_for(M, qt, flow, P.solid_scheme, (long long)P.nx * P.ny, form);
}

// L2 prefetch distance of the node-pair kernel in rows (0: off): grids of at
// least kPrefetchMinNodes nodes, whose state is far larger than L2, prefetch
// each block's chunk rows this far ahead, past most of the blocks resident at
// the same time.  One node per thread takes no prefetch: in FP32 it already
// runs at the copy bandwidth, and the extra requests slowed it down.
constexpr long long kPrefetchMinNodes = 3ll << 19;
constexpr int kPrefetchRowsPairs = 48;

inline int prefetch_rows_for(int mode, int qt, int flow, int solid_scheme, long long nodes, int form) {
    if (nodes < kPrefetchMinNodes) return 0;
    return form_for(mode, qt, flow, solid_scheme, nodes, form) == FORM_PAIRS ? kPrefetchRowsPairs : 0;
}

// The step kernel of a run, with its grid: one node per thread in blocks of
// b threads, or node pairs in blocks of 32 x 4.
struct StepLaunch {
    const void* fn;
    dim3 grid, block;
};

template <int M>
StepLaunch step_launch(const StepParams<typename ModeTraits<M>::R>& P, int qt, int flow, int form, dim3 b) {
    StepLaunch L{nullptr, dim3(), b};
    if constexpr (M != MODE_F64) {
        if (form_of<M>(P, qt, flow, form) == FORM_PAIRS) {
            L.fn = P.phase_k ? (const void*)fused_step_pair<M, true> : (const void*)fused_step_pair<M, false>;
            L.block = dim3(32, 4);   // 2048^2 FP16 61.25 us per step (64 x 2: 61.98)
            L.grid = dim3((unsigned)(((P.nx + 1) / 2 + 31) / 32), (unsigned)((P.ny + 3) / 4), 1u);
            return L;
        }
    }
    dispatch_step<M>(qt, flow, P.phase_k, [&]<int MM, int Q, bool F, bool PH>() {
        L.fn = (const void*)fused_step<MM, Q, F, PH>;
        return cudaSuccess;
    });
    L.grid = dim3((unsigned)((P.nx + b.x - 1) / b.x), (unsigned)((P.ny + b.y - 1) / b.y), 1u);
    return L;
}

// Grouped launches (map 4 of a batch): runs below kGroupMaxNodes nodes share
// grouped launches; larger runs, whose own step kernel fills the device,
// keep it (a chain of their own, as under map 3).
constexpr long long kGroupMaxNodes = 1ll << 20;

// The tile of a run in a grouped launch: the narrowest waste of threads among
// tiles 32, 64 and 128 nodes wide (ties to the wider); the idle fraction of the
// covered columns, (cover - nx) / cover, compared exactly.
inline int group_tile(int nx) {
    int best = 2;
    long long best_cover = ((nx + 127) / 128) * 128ll;
    for (int k = 1; k >= 0; --k) {
        const int w = 32 << k;
        const long long cover = (long long)((nx + w - 1) / w) * w;
        if ((cover - nx) * best_cover < (best_cover - nx) * cover) {
            best = k;
            best_cover = cover;
        }
    }
    return best;
}

// Blocks of one run in a grouped launch (blocks of 128 threads).
inline long long group_blocks(int nx, int ny, int tile) {
    const int w = 32 << tile;
    return (long long)((nx + w - 1) / w) * ((ny + (128 / w) - 1) / (128 / w));
}

template <int M>
const void* group_kernel(int qt, int flow, int ph) {
    const void* fn = nullptr;
    dispatch_step<M>(qt, flow, ph, [&]<int MM, int Q, bool F, bool PH>() {
        fn = (const void*)group_step<MM, Q, F, PH>;
        return cudaSuccess;
    });
    return fn;
}

// Launched as a programmatic dependent of the previous step (the kernels wait
// for it before touching the state), so the launch overlaps its tail.
template <int M>
cudaError_t launch_step(const StepParams<typename ModeTraits<M>::R>& P, int qt, int flow, int form, cudaStream_t s) {
    const StepLaunch L = step_launch<M>(P, qt, flow, form, step_block(P.nx, P.ny));
    void* args[1] = {const_cast<StepParams<typename ModeTraits<M>::R>*>(&P)};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = L.grid;
    cfg.blockDim = L.block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, L.fn, args);
}

// Block height of the two-step kernel (blocks of kT2W x H threads, inner
// tiles of (kT2W - 2) x (H - 2) nodes) for an nx x ny grid on nsm SMs.  Among
// the heights that leave at most two tiles per SM, the one whose busiest SM
// runs the fewest node updates (its tiles, rounded up over the SMs, times the
// block's warps for the first step and the inner tile for the second), with
// the work of two tiles per SM counted at kT2Overlap: two resident blocks
// overlap each other's L2 loads and barrier.  On 152 SMs: 128^2 takes H = 6
// (128 tiles), 192^2 H = 10 (144), 256^2 H = 9 (296; FP32 2.04 against 2.21 us
// per step for H = 16 and one tile per SM).  Grids that need more than two
// tiles per SM take H = kT2HMany = 12, measured fastest there (FP32: three
// resident blocks of 13 warps per SM; 1024^2 and 2048^2 against H = 6, 8,
// 10, 14, 16).
constexpr double kT2Overlap = 0.87;

inline long long t2_tiles(int n, int inner) { return t2_count(n, inner); }

inline dim3 t2_grid(int nx, int ny, int h) {
    return dim3((unsigned)t2_tiles(nx, kT2W - 2), (unsigned)t2_tiles(ny, h - 2), 1u);
}

inline int t2_block(int nx, int ny, int nsm) {
    if (nsm < 1) nsm = 1;
    int best = kT2HMany;
    double best_cost = -1.0;
    for (int h = 4; h <= kT2H; ++h) {
        const long long tiles = t2_tiles(nx, kT2W - 2) * t2_tiles(ny, h - 2);
        const long long per_sm = (tiles + nsm - 1) / nsm;
        if (per_sm > 2) continue;
        const long long work = per_sm * ((kT2W * h + 31) / 32 * 32 + (long long)(kT2W - 2) * (h - 2));
        const double cost = per_sm > 1 ? kT2Overlap * (double)work : (double)work;
        if (best_cost < 0.0 || cost < best_cost) {
            best = h;
            best_cost = cost;
        }
    }
    return best;
}

// The build of the kernel for block height h (h == kT2HMany: the many-tiles
// build) and its dynamic shared memory.
template <int M, int HM>
const void* step2_kernel_hm(int qt, int phase_k) {
    if (qt == 5) return phase_k ? (const void*)fused_step2<M, 5, true, HM> : (const void*)fused_step2<M, 5, false, HM>;
    return phase_k ? (const void*)fused_step2<M, 9, true, HM> : (const void*)fused_step2<M, 9, false, HM>;
}

template <int M>
const void* step2_kernel(int qt, int phase_k, int h) {
    if constexpr (M != MODE_F64) {
        return h == kT2HMany ? step2_kernel_hm<M, kT2HMany>(qt, phase_k) : step2_kernel_hm<M, kT2H>(qt, phase_k);
    }
    return nullptr;
}

template <int M>
size_t step2_smem(int qt, int h) {
    if constexpr (M != MODE_F64) {
        if (h == kT2HMany) return qt == 5 ? Tile2<M, 5, kT2HMany>::bytes : Tile2<M, 9, kT2HMany>::bytes;
        return qt == 5 ? Tile2<M, 5, kT2H>::bytes : Tile2<M, 9, kT2H>::bytes;
    }
    return 0;
}

// Batch map 5: the grouped two-step kernel and its shared memory (the 12-row
// build; blocks of kT2W x kT2HMany threads).
template <int M>
const void* group2_kernel(int qt, int phase_k) {
    if constexpr (M != MODE_F64) {
        if (qt == 5) return phase_k ? (const void*)group_step2<M, 5, true> : (const void*)group_step2<M, 5, false>;
        return phase_k ? (const void*)group_step2<M, 9, true> : (const void*)group_step2<M, 9, false>;
    }
    return nullptr;
}

inline long long group2_blocks(int nx, int ny) { return t2_tiles(nx, kT2W - 2) * t2_tiles(ny, kT2HMany - 2); }

// Two steps from copy P.src to P.dst, history P.dT -> P.dT_out, in blocks of
// kT2W x h threads, as a programmatic dependent of the previous launch in the
// stream.
template <int M>
cudaError_t launch_step2(const StepParams<typename ModeTraits<M>::R>& P, int qt, int h, cudaStream_t s) {
    if (h < 4 || h > kT2H) return cudaErrorInvalidConfiguration;
    const void* fn = step2_kernel<M>(qt, P.phase_k, h);
    if (!fn) return cudaErrorInvalidConfiguration;
    const size_t smem = step2_smem<M>(qt, h);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* args[1] = {const_cast<StepParams<typename ModeTraits<M>::R>*>(&P)};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = t2_grid(P.nx, P.ny, h);
    cfg.blockDim = dim3((unsigned)kT2W, (unsigned)h, 1u);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
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
cudaError_t launch_convert(const StepParams<typename ModeTraits<M>::R>& P,
                           const DenseState<typename ModeTraits<M>::R>& D, int to_dense, int qt, int flow,
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


template <int M>
int batch_blocks_per_sm(int qt, int flow, int ph) {
    int n = 0;
    dispatch_step<M>(qt, flow, ph, [&]<int MM, int Q, bool F, bool PH>() {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step<MM, Q, F, PH>, 256, 0);
    });
    return n;
}

// Explicit instantiations of the launchers (KW empty: in the kernel units) and
// the matching declarations (KW = extern: in the units that call them, so
// that the kernels are compiled once, in their own units).
#define LBMK_TEMPLATES(KW, M)                                                                                 \
    KW template cudaError_t launch_step<M>(const StepParams<ModeTraits<M>::R>&, int, int, int, cudaStream_t);   \
    KW template cudaError_t launch_fields<M>(const StepParams<ModeTraits<M>::R>&, const FieldOut<ModeTraits<M>::R>&, \
                                          int, int, cudaStream_t);                                            \
    KW template cudaError_t launch_diag<M>(const StepParams<ModeTraits<M>::R>&, const DiagConst&, double*, double*, \
                                        int, int, cudaStream_t);                                              \
    KW template cudaError_t launch_init<M>(const StepParams<ModeTraits<M>::R>&, const InitVals&, int, int, cudaStream_t); \
    KW template cudaError_t launch_batch<M>(const StepParams<ModeTraits<M>::R>*, const Tile*, int, int, int, int, int, \
                                         int, int, cudaStream_t);                                               \
    KW template int batch_blocks_per_sm<M>(int, int, int);                                                   \
    KW template const void* group_kernel<M>(int, int, int);                                                    \
    KW template cudaError_t launch_step2<M>(const StepParams<ModeTraits<M>::R>&, int, int, cudaStream_t);     \
    KW template const void* group2_kernel<M>(int, int);                                                        \
    KW template size_t step2_smem<M>(int, int);                                                                \
    KW template StepLaunch step_launch<M>(const StepParams<ModeTraits<M>::R>&, int, int, int, dim3);

#define LBMK_CONVERT_TEMPLATES(KW, M)                                                                         \
    KW template cudaError_t launch_convert<M>(const StepParams<ModeTraits<M>::R>&, const DenseState<ModeTraits<M>::R>&, \
                                           int, int, int, cudaStream_t);


#define LBMK_INSTANTIATE(M) LBMK_TEMPLATES(, M)
#define LBMK_INSTANTIATE_CONVERT(M) LBMK_CONVERT_TEMPLATES(, M)
#define LBMK_EXTERN(M) LBMK_TEMPLATES(extern, M) LBMK_CONVERT_TEMPLATES(extern, M)

}  // namespace lbmk
