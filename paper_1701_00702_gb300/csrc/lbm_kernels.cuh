// Device code of the fused three-lattice time step (Liu, He & Li, arXiv
// 1701.00702, Sec. III).  One thread owns one node (fused_step) or two
// neighbouring nodes (fused_step_pair); the whole step is one pass over HBM:
// 9 + 2*Q_T populations and the exchange history are read once (pull
// streaming, Eqs. 15, 33, 44) and written once.
//
// Everything after the pull works in moment space:
//   * m+ = M f+, n_g = M g, n_h = M h with the integer matrices of Eq. 13
//     (D2Q9) and Eq. B1 (D2Q5), hand-unrolled;
//   * flow populations are stored as deviations f_i - w_i from the rest
//     equilibrium f^eq(rho_0 = 1, 0) = w_i (Eq. 27), an exact change of
//     variables that keeps storage resolution proportional to u instead of
//     rho; all flow moments below are deviations from r = M w = (1, -2, 1,
//     0, ..., 0) and delta_rho = rho - 1;
//   * the volumetric blend f = f_l f+ + (1 - f_l) f^eq(rho, 0) (Eq. 20) is
//     linear, and M f^eq(rho, 0) = rho r (Eq. 18 at u = 0), so in deviation
//     form m - r = f_l (m+ - r) + (1 - f_l) delta_rho r;
//   * the wall rule of Eq. 52 is linear too: m+(x_b) = m+(x_f) +
//     m^eq(rho_f, u_b = 0) - m^eq(rho_f, u_f), and likewise for the thermal
//     moments with their own equilibria (Eqs. 34/B2, 45/B4);
//   * the collisions are Eq. 14 (flow, with forcing Eq. 19), Eq. 32 (PCM,
//     source Eqs. 35-36 or App. B) and Eq. 43 (metal, Eqs. 46-47 or App. B),
//     followed by f* = M^-1 m*, with M^-1 = M^T diag(1/|row|^2) for D2Q9;
//   * the PCM enthalpy is bookkept exactly: with FP32 storage the rest
//     population g_0 is kept as an unevaluated float-float sum (hi in the
//     g_0 plane, lo in one extra plane), H = g_0 + sum_{i>=1} g_i is formed
//     as a compensated sum of error-free additions (Knuth's TwoSum, Dekker's
//     Fast2Sum), and the post-collision rest population is the remainder
//     g_0* = n_0* - sum_{i>=1} g_i* of the stored moving populations, so that
//     streaming and collision conserve the enthalpy to ~2^-46 instead of
//     accumulating FP32 rounding in the isothermal mushy zone, where nothing
//     damps it;
//   * every other rest population is a remainder as well, and the PCM's
//     exchange source is the opposite of the change the metal's n_0 actually
//     took (scaled by the heat capacities), so the exchange moves no energy
//     that the metal's rounding dropped;
//   * the state is chunked: [chunk][plane][kChunk] with chunks of kChunk nodes
//     along x, so one pointer per pulled neighbour reaches all its planes;
//   * FP32 arithmetic goes through the packed two-lane instructions of sm_100
//     and later wherever two values take the same operations (the PCM and
//     metal lattices, pairs of flow moments, or the two nodes of a pair).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbmk {

// Storage modes.  Arithmetic is FP64 for MODE_F64 and FP32 otherwise.
//   MODE_F64  every population in FP64;
//   MODE_F32  every population in FP32, the PCM rest population as a
//             float-float pair (one extra FP32 plane for the low part);
//   MODE_F16, MODE_BF16  flow deviations (scaled by 2^10 for FP16) and the
//             moving thermal populations in 16 bits, the two thermal rest
//             populations and the exchange history in FP32.  A moving thermal
//             population is stored as its deviation from a reference that any
//             reader rebuilds from the FP32 rest population of the node that
//             sent it: at equilibrium with u = 0 every moving population is
//             w'_i c_ref T and the rest population is g_0 = H - omega c_ref T
//             (Eqs. 40, 49, B3, B5), a monotone map of the node's state, so
//             T (hence the reference) follows from g_0 alone.  The 16-bit
//             values then carry only the flux and non-equilibrium parts, and
//             the sender stores the rest population that closes the balance
//             with the movers as readers decode them.
enum : int { MODE_F64 = 0, MODE_F32 = 1, MODE_F16 = 2, MODE_BF16 = 3 };

template <int M> struct ModeTraits;
template <> struct ModeTraits<MODE_F64> { using R = double; using B = double; };
template <> struct ModeTraits<MODE_F32> { using R = float; using B = float; };
template <> struct ModeTraits<MODE_F16> { using R = float; using B = __half; };
template <> struct ModeTraits<MODE_BF16> { using R = float; using B = __nv_bfloat16; };

template <int M> constexpr bool kSplit = (M == MODE_F16 || M == MODE_BF16);
// FP16 stores the flow deviations times 2^10 (|f_i - w_i| < 1 while |u| < 0.3
// keeps them in the normal range); the other modes store them as they are.
template <int M> constexpr int kFlowScale = (M == MODE_F16) ? 1024 : 1;
template <int M> constexpr bool kComp = (M == MODE_F32);

__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ double to_f(double v) { return v; }

template <typename B> __device__ __forceinline__ B from_f(float v);
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <typename B> __device__ __forceinline__ B from_f(double v) { return v; }

// Plane numbering inside one state copy.  Bulk planes hold type B; the wide
// planes (16-bit modes only) hold the PCM (0) and metal (1) rest populations.
template <int M, int QT, bool FLOW>
struct Planes {
    static constexpr int fb = FLOW ? 9 : 0;
    __host__ __device__ static constexpr int pcm(int q) { return kSplit<M> ? fb + q - 1 : fb + q; }   // q >= 1 when split
    __host__ __device__ static constexpr int met(int q) { return kSplit<M> ? fb + (QT - 1) + q - 1 : fb + QT + q; }
    static constexpr int lo = fb + 2 * QT;                                                  // MODE_F32 only
    static constexpr int bulk = kSplit<M> ? fb + 2 * (QT - 1) : fb + 2 * QT + (kComp<M> ? 1 : 0);
    static constexpr int wide = kSplit<M> ? 2 : 0;
};

// State layout: each row is cut into chunks of kChunk nodes along x, and a
// chunk holds every plane of its nodes, [chunk][plane][kChunk]: the bulk
// planes (the mode's storage type), then the wide planes (FP32).  A node's
// element in plane q lies kChunk * q elements after its element in plane 0,
// so one pointer per pulled neighbour reaches all of that neighbour's planes
// through constant offsets.  Chunk y * cpr + x / kChunk holds node (x, y).
constexpr int kChunk = 128;
constexpr int kChunkShift = 7;

template <int M, int QT, bool FLOW>
struct Chunk {
    using B = typename ModeTraits<M>::B;
    using PL = Planes<M, QT, FLOW>;
    static constexpr int wide_off = PL::bulk * kChunk * (int)sizeof(B);        // bytes to wide plane 0
    static constexpr int bytes = wide_off + PL::wide * kChunk * (int)sizeof(float);
};

// A pair of values that go through the same arithmetic: the PCM and metal
// lattices' populations and moments (x: PCM, y: metal).  With FP32 arithmetic
// a pair operation is one packed instruction (the .f32x2 add, multiply and
// fused multiply-add of sm_100 and later), which halves the issue slots of
// that arithmetic; FP64 keeps two scalar operations.  Each lane is rounded as
// the scalar operation would be.
template <typename R>
struct alignas(2 * sizeof(R)) V2 {
    R x, y;
};

template <typename R>
__device__ __forceinline__ V2<R> add2(V2<R> a, V2<R> b) {
    if constexpr (sizeof(R) == 4) {
        const float2 r = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
        return {r.x, r.y};
    } else {
        return {a.x + b.x, a.y + b.y};
    }
}

template <typename R>
__device__ __forceinline__ V2<R> mul2(V2<R> a, V2<R> b) {
    if constexpr (sizeof(R) == 4) {
        const float2 r = __fmul2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
        return {r.x, r.y};
    } else {
        return {a.x * b.x, a.y * b.y};
    }
}

template <typename R>
__device__ __forceinline__ V2<R> fma2(V2<R> a, V2<R> b, V2<R> c) {   // a b + c, one rounding per lane
    if constexpr (sizeof(R) == 4) {
        const float2 r = __ffma2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y), make_float2(c.x, c.y));
        return {r.x, r.y};
    } else {
        return {fma(a.x, b.x, c.x), fma(a.y, b.y, c.y)};
    }
}

template <typename R>
__device__ __forceinline__ V2<R> sub2(V2<R> a, V2<R> b) {   // a - b, one rounding per lane
    return fma2(b, V2<R>{R(-1), R(-1)}, a);
}

// Per-run constants, passed by value (__grid_constant__).
template <typename R>
struct StepParams {
    const char* src;     // current state copy, [chunk][plane][kChunk]
    char* dst;           // next state copy
    R* dT;               // [ny][pitch] exchange history T_m - T_f of the previous step
    R* dT_out;           // two-step kernel: the history after its second step (another array)
    unsigned int* status;
    int nx, ny, pitch;   // pitch = cpr * kChunk
    int cpr;             // chunks per row
    int per_x, per_y;
    int solid_scheme;    // 0: volumetric blend; 1: bounce-back where f_l <= 0.5 (Sec. V B)
    int prefetch_rows;   // > 0: each block asks L2 for its chunk this many rows ahead
    int wall_kind[4];
    R wall_T[4], wall_T_lo[4], wall_H[4], wall_H_lo[4];
    R fscale, finv;      // flow deviations are stored times fscale (a power of two)
    // 16-bit modes: references of the moving thermal populations
    R w_move[9];         // w'_i: the equilibrium weight of mover i (D2Q9 w_i, D2Q5 varpi/4)
    R g0_fs, g0_fl;      // PCM rest population at solidus / liquidus equilibrium
    R cr_solid, cr_liquid;   // c_f,ref dT/dg_0 on the solid and liquid branches
    R cr_fs, cr_dsl;     // c_f,ref T_fs, c_f,ref (T_fl - T_fs)
    R inv_dg0;           // 1 / (g0_fl - g0_fs)
    R wk_move[9];        // w'_i kappa_m: metal mover reference per unit of h_0
    R kappa_m;           // c_m,ref / (c_pm - omega c_m,ref): mover reference per unit of h_0 / w'_i
    R om_cf;             // omega c_f,ref (omega = sum of the w'_i): g_0 = H - om_cf T(H) at equilibrium
    R rest_m;            // 1 - omega c_m,ref / c_pm: h_0 = rest_m c_pm T_m at equilibrium
    // flow (Eqs. 3, 7, 16, 25)
    R phi, inv_phi, drag_lin, drag_forch, gbeta, T0, l0, l0sq, l1;
    R s[9];
    // thermal (Eqs. 38-39, 34, 45, App. B)
    // (c_pl = c_pm = 1 in the lattice units of Eq. 54, so they appear nowhere below)
    R H_fs, H_fl, inv_dH, T_fs, T_fl, dT_sl, inv_c_ps;   // dT_sl = T_fl - T_fs
    R c_fref, c_mref, varpi;
    R vcf, vcm;          // varpi c_f,ref and varpi c_m,ref (D2Q5 equilibria, Eqs. B2, B4)
    R eta[9];            // metal rates (eta[0] for the FP32 rest population's relaxation)
    V2<R> nrate[9];      // (-zeta_k, -eta_k): PCM and metal relaxation rates, negated
    V2<R> nwmv[9];       // (-w'_k, -w'_k kappa_m): 16-bit mover references per unit of (ref, h_0)
    V2<R> wmv[9];        // (w'_k, w'_k kappa_m)
    R a_m;               // h_v/((1 - phi) rho_m), Eq. 47
    R x_pm;              // -a_f/a_m = -(1 - phi) rho_m/(phi rho_l): PCM source per unit of metal source
    // Eq. 9 variant: PCM rates from the node's liquid fraction
    int phase_k;         // 1: k_s != k_l, rates per node
    R kl_c, ks_c;        // k_l, k_s over (rho_l c_fref c_sT^2)
    R zr_a[9], zr_b[9];  // PCM rate k = zr_a[k] + zr_b[k] zeta_alpha
};

enum : unsigned int { STATUS_UNSTABLE = 1u };

// Error-free transformations (IEEE round-to-nearest, no contraction).
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF two_sum(float a, float b) {        // Knuth
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ FF fast_two_sum(float a, float b) {   // Dekker, |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ FF ff_add(FF a, float b) {
    const FF s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}


// a.hi + a.lo + sign * (v[1] + ... + v[Q-1]) as a float-float pair: each term
// enters through TwoSum, the rounding errors gather in one float, and the pair
// is normalised once at the end (a compensated sum; its error is of the order
// of (Q - 1) u^2 |sum|, u = 2^-24).
template <int Q>
__device__ __forceinline__ FF ff_accumulate(FF a, const float* v, float sign) {
    float s = a.hi, c = a.lo;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const FF t = two_sum(s, sign * v[i]);
        s = t.hi;
        c = __fadd_rn(c, t.lo);
    }
    return fast_two_sum(s, c);
}

// ---------------------------------------------------------------------------
// Transforms
// ---------------------------------------------------------------------------

template <typename R>
__device__ __forceinline__ void m_from_f9(const R* f, R* m) {
    const R s14 = f[1] + f[2] + f[3] + f[4];
    const R s58 = f[5] + f[6] + f[7] + f[8];
    const R dx = f[1] - f[3], dy = f[2] - f[4];
    const R ax = f[5] - f[6] - f[7] + f[8];
    const R ay = f[5] + f[6] - f[7] - f[8];
    m[0] = f[0] + s14 + s58;
    m[1] = R(-4) * f[0] - s14 + R(2) * s58;
    m[2] = R(4) * f[0] - R(2) * s14 + s58;
    m[3] = dx + ax;
    m[4] = R(-2) * dx + ax;
    m[5] = dy + ay;
    m[6] = R(-2) * dy + ay;
    m[7] = f[1] - f[2] + f[3] - f[4];
    m[8] = f[5] - f[6] + f[7] - f[8];
}

// f = M^-1 m, every f scaled by SC (a power of two: the 16-bit flow storage
// scale, folded into the row norms).
template <typename R, int SC = 1>
__device__ __forceinline__ void f_from_m9(const R* m, R* f) {
    constexpr double s = SC;
    const R A = m[0] * R(s / 9.0), B = m[1] * R(s / 36.0), C = m[2] * R(s / 36.0);
    const R DX = m[3] * R(s / 6.0), QX = m[4] * R(s / 12.0);
    const R DY = m[5] * R(s / 6.0), QY = m[6] * R(s / 12.0);
    const R P = m[7] * R(s * 0.25), S = m[8] * R(s * 0.25);
    f[0] = A - R(4) * B + R(4) * C;
    const R b1 = A - B - R(2) * C;
    f[1] = b1 + DX - R(2) * QX + P;
    f[3] = b1 - DX + R(2) * QX + P;
    f[2] = b1 + DY - R(2) * QY - P;
    f[4] = b1 - DY + R(2) * QY - P;
    const R b5 = A + R(2) * B + C;
    const R X = DX + QX, Y = DY + QY;
    f[5] = b5 + X + Y + S;
    f[6] = b5 - X + Y - S;
    f[7] = b5 - X - Y + S;
    f[8] = b5 + X - Y - S;
}

// Eq. 13 on the population pairs (f1, f2), (f3, f4), (f5, f6), (f7, f8) (the
// D2Q9 order of Eq. 11): m_0 and the moment pairs (e, eps), (j_x, j_y),
// (q_x, q_y), (p_xx, p_xy).
template <typename R>
__device__ __forceinline__ void m_from_f9p(R f0, const V2<R>* F, R& m0, V2<R>* m) {
    const V2<R> A = add2(F[0], F[1]);   // (f1 + f3, f2 + f4)
    const V2<R> D = sub2(F[0], F[1]);   // (f1 - f3, f2 - f4)
    const V2<R> B = add2(F[2], F[3]);   // (f5 + f7, f6 + f8)
    const V2<R> E = sub2(F[2], F[3]);   // (f5 - f7, f6 - f8)
    const R s14 = A.x + A.y, s58 = B.x + B.y;
    const V2<R> a = {E.x - E.y, E.x + E.y};   // (f5 - f6 - f7 + f8, f5 + f6 - f7 - f8)
    m0 = f0 + s14 + s58;
    m[0] = {R(-4) * f0 - s14 + R(2) * s58, R(4) * f0 - R(2) * s14 + s58};
    m[1] = add2(D, a);
    m[2] = fma2(V2<R>{R(-2), R(-2)}, D, a);
    m[3] = {A.x - A.y, B.x - B.y};
}

// f = M^-1 m on the same pairs, every f scaled by SC (as f_from_m9).
template <typename R, int SC = 1>
__device__ __forceinline__ void f_from_m9p(R m0, const V2<R>* m, R& f0, V2<R>* F) {
    constexpr double s = SC;
    const R A = m0 * R(s / 9.0);
    const V2<R> BC = mul2(m[0], V2<R>{R(s / 36.0), R(s / 36.0)});   // (B, C)
    const V2<R> D = mul2(m[1], V2<R>{R(s / 6.0), R(s / 6.0)});      // (DX, DY)
    const V2<R> Q = mul2(m[2], V2<R>{R(s / 12.0), R(s / 12.0)});    // (QX, QY)
    const V2<R> PS = mul2(m[3], V2<R>{R(s * 0.25), R(s * 0.25)});   // (P, S)
    f0 = A - R(4) * BC.x + R(4) * BC.y;
    const R b1 = A - BC.x - R(2) * BC.y;
    const R b5 = A + R(2) * BC.x + BC.y;
    const V2<R> T = fma2(V2<R>{R(-2), R(-2)}, Q, D);   // (DX - 2 QX, DY - 2 QY)
    const V2<R> X = add2(D, Q);                         // (DX + QX, DY + QY)
    const V2<R> bp = {b1 + PS.x, b1 - PS.x};
    F[0] = add2(bp, T);                                 // (f1, f2)
    F[1] = sub2(bp, T);                                 // (f3, f4)
    const V2<R> G = {b5 + PS.y, b5 - PS.y}, H = {X.x + X.y, X.y - X.x};
    F[2] = add2(G, H);                                  // (f5, f6)
    F[3] = sub2(G, H);                                  // (f7, f8)
}

// Eq. B1 and its inverse on (PCM, metal) pairs: n = M g for D2Q5 with
// n_0 = g_0 + ((g_1 + g_3) + (g_2 + g_4)), n_1 = g_1 - g_3, n_2 = g_2 - g_4,
// n_3 = g_1 + g_2 + g_3 + g_4, n_4 = g_1 - g_2 + g_3 - g_4.
template <typename R>
__device__ __forceinline__ void m_from_f5(const V2<R>* g, V2<R>* n) {
    const V2<R> a = add2(g[1], g[3]), b = add2(g[2], g[4]);
    n[1] = sub2(g[1], g[3]);
    n[2] = sub2(g[2], g[4]);
    n[3] = add2(a, b);
    n[4] = sub2(a, b);
    n[0] = add2(g[0], n[3]);
}

template <typename R>
__device__ __forceinline__ void f_from_m5(const V2<R>* n, V2<R>* g) {
    const V2<R> qu = {R(0.25), R(0.25)}, h = {R(0.5), R(0.5)}, mh = {R(-0.5), R(-0.5)};
    const V2<R> p = mul2(add2(n[3], n[4]), qu), q = mul2(sub2(n[3], n[4]), qu);
    g[0] = sub2(n[0], n[3]);
    g[1] = fma2(h, n[1], p);
    g[3] = fma2(mh, n[1], p);
    g[2] = fma2(h, n[2], q);
    g[4] = fma2(mh, n[2], q);
}

template <typename R, int Q>
__device__ __forceinline__ void fwd2(const V2<R>* v, V2<R>* m) {
    if constexpr (Q == 5) {
        m_from_f5(v, m);
    } else {
        R a[9], b[9], ma[9], mb[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) { a[k] = v[k].x; b[k] = v[k].y; }
        m_from_f9(a, ma);
        m_from_f9(b, mb);
#pragma unroll
        for (int k = 0; k < 9; ++k) m[k] = {ma[k], mb[k]};
    }
}

template <typename R, int Q>
__device__ __forceinline__ void inv2(const V2<R>* m, V2<R>* v) {
    if constexpr (Q == 5) {
        f_from_m5(m, v);
    } else {
        R a[9], b[9], va[9], vb[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) { a[k] = m[k].x; b[k] = m[k].y; }
        f_from_m9(a, va);
        f_from_m9(b, vb);
#pragma unroll
        for (int k = 0; k < 9; ++k) v[k] = {va[k], vb[k]};
    }
}

// ---------------------------------------------------------------------------
// Equilibrium moments
// ---------------------------------------------------------------------------

// Eq. 34 (D2Q9) / Eq. B2 (D2Q5)
template <typename R, int Q>
__device__ __forceinline__ void neq_pcm(const StepParams<R>& P, R H, R T, R ux, R uy, R* ne) {
    const R t = T * P.inv_phi;   // c_pl T / phi
    const R jx = t * ux, jy = t * uy;
    if constexpr (Q == 9) {
        ne[0] = H;
        ne[1] = R(-4) * H + R(2) * P.c_fref * T;
        ne[2] = R(4) * H - R(3) * P.c_fref * T;
        ne[3] = jx; ne[4] = -jx; ne[5] = jy; ne[6] = -jy;
        ne[7] = R(0); ne[8] = R(0);
    } else {
        ne[0] = H; ne[1] = jx; ne[2] = jy; ne[3] = P.vcf * T; ne[4] = R(0);
    }
}

// Eq. 45 (D2Q9) / Eq. B4 (D2Q5)
template <typename R, int Q>
__device__ __forceinline__ void neq_metal(const StepParams<R>& P, R Tm, R* ne) {
    if constexpr (Q == 9) {
        const R e = Tm;   // c_pm T_m
        ne[0] = e;
        ne[1] = R(-4) * e + R(2) * P.c_mref * Tm;
        ne[2] = R(4) * e - R(3) * P.c_mref * Tm;
#pragma unroll
        for (int k = 3; k < 9; ++k) ne[k] = R(0);
    } else {
        ne[0] = Tm; ne[1] = R(0); ne[2] = R(0); ne[3] = P.vcm * Tm; ne[4] = R(0);   // ne[0] = c_pm T_m
    }
}

template <typename R>
__device__ __forceinline__ R sat01(R x) {
    if constexpr (sizeof(R) == 4) return __saturatef(x);
    else return fmin(fmax(x, R(0)), R(1));
}

// Eqs. 38-39 without branches: f_l = clamp((H - H_s)/(H_l - H_s), 0, 1) and
// T = min(H/c_ps, T_s) + f_l (T_l - T_s) + max(H - H_l, 0)/c_pl, which is
// H/c_ps below the solidus, T_s + f_l (T_l - T_s) in the mushy zone and
// T_l + (H - H_l)/c_pl above the liquidus (c_pl = 1).
template <typename R>
__device__ __forceinline__ void enthalpy_state(const StepParams<R>& P, R H, R& T, R& fl) {
    fl = sat01((H - P.H_fs) * P.inv_dH);
    T = fmin(H * P.inv_c_ps, P.T_fs) + fl * P.dT_sl + fmax(H - P.H_fl, R(0));
}

// c_f,ref T at equilibrium as a function of the PCM rest population g_0: the
// inverse of g_0 = H - omega c_f,ref T(H) with T(H) from Eq. 38 (16-bit modes).
template <typename R>
__device__ __forceinline__ R pcm_ref(const StepParams<R>& P, R g0) {
    // the three branches as in enthalpy_state: solid slope up to g0_fs, a linear
    // rise of c_f,ref (T_fl - T_fs) across the mushy zone, liquid slope above g0_fl
    return fmin(g0 * P.cr_solid, P.cr_fs) + sat01((g0 - P.g0_fs) * P.inv_dg0) * P.cr_dsl +
           fmax(g0 - P.g0_fl, R(0)) * P.cr_liquid;
}

template <typename R>
__device__ __forceinline__ R fast_rcp(R x) {
    if constexpr (sizeof(R) == 4) return __fdividef(1.0f, x);
    else return R(1) / x;
}

template <typename R>
__device__ __forceinline__ R fast_sqrt(R x) {   // x >= 0
    if constexpr (sizeof(R) == 4) return x > 0.0f ? x * rsqrtf(x) : 0.0f;
    else return sqrt(x);
}

// ---------------------------------------------------------------------------
// Node state
// ---------------------------------------------------------------------------

template <int M, int QT, bool FLOW>
struct NodeState {
    using R = typename ModeTraits<M>::R;
    R mp[FLOW ? 9 : 1];  // moments of f+ minus r (after the wall rule)
    V2<R> th[QT];        // moments of (g, h) (after the wall rule); th[0] = (H, c_pm T_m) (high parts)
    R Hlo, Elo;          // low parts of H and c_pm T_m (error-free bookkeeping; 0 where unused)
    R H, Tf, fl, Tm, rho, drho, ux, uy, um, Gy;   // um = |u|
};

template <int M>
__device__ __forceinline__ typename ModeTraits<M>::R ldb(const typename ModeTraits<M>::B* p) {
    return to_f(__ldg(p));
}

template <int M, typename R>
__device__ __forceinline__ void stb(typename ModeTraits<M>::B* p, R v) {
    using B = typename ModeTraits<M>::B;
    *p = from_f<B>(v);
}

// The nine flow populations of one node (f_0 and the pairs of f_from_m9p);
// PS: elements from one plane to the next (kChunk in a state copy, where the
// inlined constant folds into the addresses).
template <int M>
__device__ __forceinline__ void store_flow(typename ModeTraits<M>::B* db, typename ModeTraits<M>::R f0,
                                           const V2<typename ModeTraits<M>::R>* F, int PS = kChunk) {
    stb<M>(db, f0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        stb<M>(db + (2 * j + 1) * PS, F[j].x);
        stb<M>(db + (2 * j + 2) * PS, F[j].y);
    }
}

// Byte offset, within a state copy, of the chunk holding node (x, y).
template <int M, int QT, bool FLOW, typename R>
__device__ __forceinline__ long long chunk_at(const StepParams<R>& P, int x, int y) {
    return (long long)(y * P.cpr + (x >> kChunkShift)) * Chunk<M, QT, FLOW>::bytes;
}

// Node (x, y)'s element in bulk plane 0 and in wide plane 0 of a copy; plane q
// follows at q * kChunk elements.
template <int M, int QT, bool FLOW, typename R, typename C>
__device__ __forceinline__ auto bulk_at(C* base, const StepParams<R>& P, int x, int y) {
    using B = typename ModeTraits<M>::B;
    using T = std::conditional_t<std::is_const_v<C>, const B, B>;
    return reinterpret_cast<T*>(base + chunk_at<M, QT, FLOW>(P, x, y)) + (x & (kChunk - 1));
}

template <int M, int QT, bool FLOW, typename R, typename C>
__device__ __forceinline__ auto wide_at(C* base, const StepParams<R>& P, int x, int y) {
    using T = std::conditional_t<std::is_const_v<C>, const float, float>;
    return reinterpret_cast<T*>(base + chunk_at<M, QT, FLOW>(P, x, y) + Chunk<M, QT, FLOW>::wide_off) +
           (x & (kChunk - 1));
}

// Byte offset of node x's element in bulk plane 0 (WIDE: wide plane 0) from
// the start of its row of chunks; a row of chunks is cpr * Chunk::bytes long
// (below 2^31 bytes for every admitted grid).
template <int M, int QT, bool FLOW, bool WIDE = false>
__device__ __forceinline__ int col_off(int x) {
    using CH = Chunk<M, QT, FLOW>;
    constexpr int es = WIDE ? (int)sizeof(float) : (int)sizeof(typename ModeTraits<M>::B);
    return (x >> kChunkShift) * CH::bytes + (WIDE ? CH::wide_off : 0) + (x & (kChunk - 1)) * es;
}

// Pull streaming around node (xs, ys): the population along e_i comes from
// xs - e_i.  The index wrap is also correct for interior nodes of a walled
// direction, which never reach the edge.  PullAt holds the addressing (one
// 64-bit row pointer per source row, one 32-bit offset per source column);
// pull_flow and pull_thermal load one side each, so that the flow and the
// thermal lattices of a node can also be pulled by two different threads.
// Source column and row (x - e_x, y - e_y) of direction q, D2Q9 order of Eq. 11,
// as 0 (x - 1 or y - 1), 1 (x or y), 2 (x + 1 or y + 1): columns 1 0 1 2 1 0 2 2 0,
// rows 1 1 0 1 2 0 0 2 2, two bits per direction.
__host__ __device__ constexpr int src_col(int q) { return (0xa191 >> (2 * q)) & 3; }
__host__ __device__ constexpr int src_row(int q) { return (0x28245 >> (2 * q)) & 3; }

template <int M, int QT, bool FLOW>
struct PullAt {
    const char* row[3];
    int dc[3];   // bulk plane 0 of source columns x - 1, x, x + 1, from this node's
    int dw[3];   // wide plane 0 of the same columns (16-bit modes)
    int xm, xs, xp, c0;
    __device__ __forceinline__ PullAt(const StepParams<typename ModeTraits<M>::R>& P, int x, int ys) : xs(x) {
        xm = xs == 0 ? P.nx - 1 : xs - 1;
        xp = xs == P.nx - 1 ? 0 : xs + 1;
        const int ym = ys == 0 ? P.ny - 1 : ys - 1;
        const int yp = ys == P.ny - 1 ? 0 : ys + 1;
        const int rb = P.cpr * Chunk<M, QT, FLOW>::bytes;
        c0 = col_off<M, QT, FLOW>(xs);
        const char* own = P.src + ((long long)ys * rb + c0);
        row[0] = own + (long long)(ym - ys) * rb;
        row[1] = own;
        row[2] = own + (long long)(yp - ys) * rb;
        dc[0] = col_off<M, QT, FLOW>(xm) - c0;
        dc[1] = 0;
        dc[2] = col_off<M, QT, FLOW>(xp) - c0;
        if constexpr (kSplit<M>) {
            dw[0] = col_off<M, QT, FLOW, true>(xm) - c0;
            dw[1] = col_off<M, QT, FLOW, true>(xs) - c0;
            dw[2] = col_off<M, QT, FLOW, true>(xp) - c0;
        }
    }
    // the source node of direction q: its element in bulk plane 0
    __device__ __forceinline__ const typename ModeTraits<M>::B* src(int q) const {
        return reinterpret_cast<const typename ModeTraits<M>::B*>(row[src_row(q)] + dc[src_col(q)]);
    }
    // bulk plane `plane` and wide plane w (16-bit modes) of the source node of direction q
    __device__ __forceinline__ typename ModeTraits<M>::R bulk(int q, int plane) const {
        return ldb<M>(src(q) + plane * kChunk);
    }
    __device__ __forceinline__ float wide(int q, int w) const {
        return __ldg(reinterpret_cast<const float*>(row[src_row(q)] + dw[src_col(q)]) + w * kChunk);
    }
};

// Flow moments of the pulled populations (Eqs. 13, 15), deviation form.  A
// is the accessor of the pulled neighbourhood: PullAt (the state copy in
// global memory) or a staged copy in shared memory.
template <int M, int QT, bool FLOW, typename A>
__device__ __forceinline__ void pull_flow(const StepParams<typename ModeTraits<M>::R>& P, const A& a,
                                          NodeState<M, QT, FLOW>& n) {
    using R = typename ModeTraits<M>::R;
    if constexpr (FLOW) {
        R f0 = a.bulk(0, 0);
        V2<R> F[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) F[j] = {a.bulk(2 * j + 1, 2 * j + 1), a.bulk(2 * j + 2, 2 * j + 2)};
        if constexpr (M == MODE_F16) {
            constexpr R is = R(1.0 / 1024.0);
            f0 *= is;
#pragma unroll
            for (int j = 0; j < 4; ++j) F[j] = mul2(F[j], V2<R>{is, is});
        }
        V2<R> m[4];
        m_from_f9p(f0, F, n.mp[0], m);
        n.mp[1] = m[0].x; n.mp[2] = m[0].y;
        n.mp[3] = m[1].x; n.mp[5] = m[1].y;
        n.mp[4] = m[2].x; n.mp[6] = m[2].y;
        n.mp[7] = m[3].x; n.mp[8] = m[3].y;
    }
}

// PCM and metal moments of the pulled populations (Eqs. 33, 44, B1).
template <int M, int QT, bool FLOW, typename A>
__device__ __forceinline__ void pull_thermal(const StepParams<typename ModeTraits<M>::R>& P, const A& a,
                                             NodeState<M, QT, FLOW>& n) {
    using R = typename ModeTraits<M>::R;
    using PL = Planes<M, QT, FLOW>;
    V2<R> t[QT];   // (g_q, h_q)
    if constexpr (kSplit<M>) {
        t[0] = {a.wide(0, 0), a.wide(0, 1)};
#pragma unroll
        for (int q = 1; q < QT; ++q) {   // deviation + reference of the sending node
            const V2<R> dev = {a.bulk(q, PL::pcm(q)), a.bulk(q, PL::met(q))};
            const V2<R> ref = {pcm_ref(P, a.wide(q, 0)), a.wide(q, 1)};
            t[q] = fma2(P.wmv[QT == 5 ? 1 : q], ref, dev);   // D2Q5: one weight varpi/4 for all movers (App. B)
        }
    } else {
#pragma unroll
        for (int q = 0; q < QT; ++q) t[q] = {a.bulk(q, PL::pcm(q)), a.bulk(q, PL::met(q))};
    }
    fwd2<R, QT>(t, n.th);
    n.Hlo = R(0);
    n.Elo = R(0);
    if constexpr (kComp<M>) {
        // H = (g_0 hi + g_0 lo) + sum of movers, without rounding loss
        const float lo = a.bulk(0, PL::lo);
        float g[QT];
#pragma unroll
        for (int q = 0; q < QT; ++q) g[q] = t[q].x;
        const FF H = ff_accumulate<QT>(FF{g[0], lo}, g, 1.0f);
        n.th[0].x = H.hi;
        n.Hlo = H.lo;
    }
}

template <int M, int QT, bool FLOW>
__device__ __forceinline__ void pull_moments(const StepParams<typename ModeTraits<M>::R>& P, int xs, int ys,
                                             NodeState<M, QT, FLOW>& n) {
    const PullAt<M, QT, FLOW> a(P, xs, ys);
    pull_flow<M, QT, FLOW>(P, a, n);
    pull_thermal<M, QT, FLOW>(P, a, n);
}

// Macroscopic state from the moments (Eqs. 21, 23-25, 37-39, 48, 7): the
// thermal side (H -> T_f, f_l; T_m) and the flow side, which needs T_f and
// f_l (buoyancy, Eq. 7; the blended momentum, Eq. 24).
template <int M, int QT, bool FLOW>
__device__ __forceinline__ void thermal_macro(const StepParams<typename ModeTraits<M>::R>& P,
                                              NodeState<M, QT, FLOW>& n) {
    n.H = n.th[0].x;
    enthalpy_state(P, n.H, n.Tf, n.fl);
    n.Tm = n.th[0].y;   // h_0 moment = c_pm T_m, c_pm = 1
}

template <int M, int QT, bool FLOW>
__device__ __forceinline__ void flow_macro(const StepParams<typename ModeTraits<M>::R>& P, NodeState<M, QT, FLOW>& n,
                                           bool wall) {
    using R = typename ModeTraits<M>::R;
    if constexpr (FLOW) {
        n.drho = n.mp[0];
        n.rho = R(1) + n.drho;
        n.Gy = P.gbeta * (n.Tf - P.T0) * n.fl;
        if (wall || (P.solid_scheme && n.fl <= R(0.5))) {
            n.ux = R(0);
            n.uy = R(0);
            n.um = R(0);
        } else {
            // Eq. 24 with sum_i e_i f_i = f_l sum_i e_i f+_i (the equilibrium at rest carries no
            // momentum); without the blend (bounce-back variant) sum_i e_i f_i = sum_i e_i f+_i
            const R ir = fast_rcp(n.rho);
            const R a = P.solid_scheme ? R(1) : n.fl;
            const R vx = a * n.mp[3] * ir;
            const R vy = a * n.mp[5] * ir + R(0.5) * P.phi * n.Gy;
            const R vm = fast_sqrt(vx * vx + vy * vy);
            const R den = fast_rcp(P.l0 + fast_sqrt(P.l0sq + P.l1 * vm));   // Eq. 23
            n.ux = vx * den;
            n.uy = vy * den;
            n.um = vm * den;
        }
    } else {
        n.drho = R(0);
        n.rho = R(1);
        n.ux = R(0);
        n.uy = R(0);
        n.um = R(0);
        n.Gy = R(0);
    }
}

template <int M, int QT, bool FLOW>
__device__ __forceinline__ void macro(const StepParams<typename ModeTraits<M>::R>& P, NodeState<M, QT, FLOW>& n,
                                      bool wall) {
    thermal_macro<M, QT, FLOW>(P, n);
    flow_macro<M, QT, FLOW>(P, n, wall);
}

// Wall nodes: x_f = x_b + inward normal (diagonal at corners) and the side
// whose temperature rule applies (the left/right wall at corners).
struct WallAt {
    bool wall;
    int xs, ys, side;
};

template <typename R>
__device__ __forceinline__ WallAt wall_at(const StepParams<R>& P, int x, int y) {
    const bool wx = !P.per_x && (x == 0 || x == P.nx - 1);
    const bool wy = !P.per_y && (y == 0 || y == P.ny - 1);
    WallAt w;
    w.wall = wx || wy;
    w.xs = wx ? (x == 0 ? 1 : P.nx - 2) : x;
    w.ys = wy ? (y == 0 ? 1 : P.ny - 2) : y;
    w.side = wx ? (x == 0 ? 0 : 1) : (y == 0 ? 2 : 3);
    return w;
}

// Eq. 52 in moment space on the flow lattice: m+(x_b) = m+(x_f) +
// m^eq(rho_f, u_b = 0) - m^eq(rho_f, u_f), written out so that the rho r
// parts cancel exactly (n holds the state of x_f).
template <int M, int QT, bool FLOW>
__device__ __forceinline__ void flow_wall(const StepParams<typename ModeTraits<M>::R>& P, NodeState<M, QT, FLOW>& n) {
    using R = typename ModeTraits<M>::R;
    if constexpr (FLOW) {
        const R rho = n.rho, ip = P.inv_phi;
        const R q = R(3) * rho * (n.ux * n.ux + n.uy * n.uy) * ip;
        n.mp[1] -= q;
        n.mp[2] += q;
        n.mp[3] -= rho * n.ux;
        n.mp[4] += rho * n.ux;
        n.mp[5] -= rho * n.uy;
        n.mp[6] += rho * n.uy;
        n.mp[7] -= rho * (n.ux * n.ux - n.uy * n.uy) * ip;
        n.mp[8] -= rho * n.ux * n.uy * ip;
    }
}

// Eq. 52 on the PCM and metal lattices, with the wall's temperature
// (Dirichlet: T_f = T_m = T_w, H = H(T_w); adiabatic: those of x_f) and the
// velocity u_f of x_f in the PCM equilibrium.
template <int M, int QT, bool FLOW>
__device__ __forceinline__ void thermal_wall(const StepParams<typename ModeTraits<M>::R>& P,
                                             NodeState<M, QT, FLOW>& n, int side) {
    using R = typename ModeTraits<M>::R;
    const bool dirichlet = P.wall_kind[side] == 0;
    R Tb, Hb, Tmb;
    if (dirichlet) {
        Tb = P.wall_T[side];
        Tmb = Tb;
        Hb = P.wall_H[side];
    } else {
        Tb = n.Tf;
        Hb = n.H;
        Tmb = n.Tm;
    }
    R a[QT], b[QT];
    neq_pcm<R, QT>(P, Hb, Tb, R(0), R(0), a);
    neq_pcm<R, QT>(P, n.H, n.Tf, n.ux, n.uy, b);
#pragma unroll
    for (int k = 1; k < QT; ++k) n.th[k].x += a[k] - b[k];
    if (dirichlet) {   // n_0 = H_b exactly (adiabatic: n_0 = H(x_f), unchanged)
        n.th[0].x = P.wall_H[side];
        n.Hlo = P.wall_H_lo[side];
    }
    neq_metal<R, QT>(P, Tmb, a);
    neq_metal<R, QT>(P, n.Tm, b);
    if constexpr (kSplit<M>) {
#pragma unroll
        for (int k = 1; k < QT; ++k) n.th[k].y += a[k] - b[k];
        if (dirichlet) {   // c_pm T_m = c_pm T_b exactly (c_pm = 1)
            n.th[0].y = P.wall_T[side];
            n.Elo = P.wall_T_lo[side];
        }
    } else {
#pragma unroll
        for (int k = 0; k < QT; ++k) n.th[k].y += a[k] - b[k];
    }
}

// State of a node from its pulled neighbourhood a (pulled at x_f on walls,
// then Eq. 52 in moment space).
template <int M, int QT, bool FLOW, typename A>
__device__ __forceinline__ void node_state_from(const StepParams<typename ModeTraits<M>::R>& P, const A& a,
                                                const WallAt& w, NodeState<M, QT, FLOW>& n) {
    pull_flow<M, QT, FLOW>(P, a, n);
    pull_thermal<M, QT, FLOW>(P, a, n);
    macro<M, QT, FLOW>(P, n, false);
    if (!w.wall) return;
    flow_wall<M, QT, FLOW>(P, n);
    thermal_wall<M, QT, FLOW>(P, n, w.side);
    macro<M, QT, FLOW>(P, n, true);
}

// Full state of node (x, y): interior nodes pull at themselves; wall nodes pull
// at x_f = x_b + inward normal and apply Eq. 52 in moment space.
template <int M, int QT, bool FLOW>
__device__ __forceinline__ void node_state(const StepParams<typename ModeTraits<M>::R>& P, int x, int y,
                                           NodeState<M, QT, FLOW>& n, bool& wall) {
    const WallAt w = wall_at(P, x, y);
    wall = w.wall;
    const PullAt<M, QT, FLOW> a(P, w.xs, w.ys);
    node_state_from<M, QT, FLOW>(P, a, w, n);
}

// Post-collision thermal populations of both lattices from their moments
// (x: PCM, y: metal).  n0g (hi, lo) and n0h are the conserved moments after the
// sources.  Each rest population is the remainder n_0 - sum of the moving
// populations as they are stored, so the stored populations carry the enthalpy
// (internal energy) that the collision produced: the FP32 PCM rest population
// to float-float accuracy, the FP32 metal one to one rounding, the 16-bit forms
// to FP32 rounding as readers decode them, FP64 to FP64 rounding.  db and dw
// point at the node's element in bulk plane 0 and wide plane 0 of the next copy
// (PS elements from one plane to the next).
template <int M, int QT, bool FLOW>
__device__ __forceinline__ void store_thermal(const StepParams<typename ModeTraits<M>::R>& P,
                                              V2<typename ModeTraits<M>::R>* nm, typename ModeTraits<M>::R n0ghi,
                                              typename ModeTraits<M>::R n0glo, typename ModeTraits<M>::R n0h,
                                              typename ModeTraits<M>::B* db, float* dw, int PS = kChunk) {
    using R = typename ModeTraits<M>::R;
    using B = typename ModeTraits<M>::B;
    using PL = Planes<M, QT, FLOW>;
    V2<R> v[QT];
    nm[0] = {n0ghi, n0h};
    inv2<R, QT>(nm, v);
    if constexpr (kSplit<M>) {
        // 16-bit deviations from the reference of the provisional rest population,
        // then the rest population readers will see the balance with.  Readers
        // rebuild the reference from the stored rest population g_0; with
        // Y = n_0 - sum of the stored deviations the balance needs
        // g_0 + omega ref(g_0) = Y, and since g_0 = H - omega c_ref T(H) is the
        // equilibrium rest population of an enthalpy H (Eqs. 38, 40, B3; Eqs. 49,
        // B5 for the metal), the solution is that of H = Y: g_0 = Y - omega
        // c_ref T(Y), whose reference is c_ref T(Y).  The stored populations as
        // read then carry n_0 to FP32 rounding.
        const V2<float> ref = {pcm_ref(P, v[0].x), v[0].y};   // v[0]: provisional rest populations
        V2<float> sd;
#pragma unroll
        for (int k = 1; k < QT; ++k) {
            const V2<float> e = fma2(P.nwmv[QT == 5 ? 1 : k], ref, v[k]);
            const B bg = from_f<B>(e.x), bh = from_f<B>(e.y);
            db[PL::pcm(k) * PS] = bg;
            db[PL::met(k) * PS] = bh;
            const V2<float> d = {to_f(bg), to_f(bh)};
            sd = k == 1 ? d : add2(sd, d);
        }
        const V2<float> Y = sub2(V2<float>{n0ghi, n0h}, sd);
        float T, fl;
        enthalpy_state(P, Y.x, T, fl);
        dw[0] = Y.x - P.om_cf * T;
        dw[PS] = Y.y * P.rest_m;
    } else {
#pragma unroll
        for (int k = 1; k < QT; ++k) {
            stb<M>(db + PL::pcm(k) * PS, v[k].x);
            stb<M>(db + PL::met(k) * PS, v[k].y);
        }
        V2<R> sm = v[1];
#pragma unroll
        for (int k = 2; k < QT; ++k) sm = add2(sm, v[k]);
        const V2<R> rest = sub2(V2<R>{n0ghi, n0h}, sm);
        if constexpr (kComp<M>) {   // the FP32 PCM rest population is a float-float pair
            float vg[QT];
#pragma unroll
            for (int k = 0; k < QT; ++k) vg[k] = v[k].x;
            const FF r = ff_accumulate<QT>(FF{n0ghi, n0glo}, vg, -1.0f);
            stb<M>(db + PL::pcm(0) * PS, r.hi);
            stb<M>(db + PL::lo * PS, r.lo);
        } else {
            stb<M>(db + PL::pcm(0) * PS, rest.x);
        }
        stb<M>(db + PL::met(0) * PS, rest.y);
    }
}

// ---------------------------------------------------------------------------
// The fused step
// ---------------------------------------------------------------------------

// Flow collision and store of one node (Eqs. 3, 14, 18-20): f* at db, this
// node's element in flow plane 0 of the next copy.
template <int M, int QT, bool FLOW>
__device__ __forceinline__ void flow_collide(const StepParams<typename ModeTraits<M>::R>& P,
                                             const NodeState<M, QT, FLOW>& n, typename ModeTraits<M>::B* db,
                                             int PS = kChunk) {
    using R = typename ModeTraits<M>::R;
    if constexpr (FLOW) {
      if (P.solid_scheme && n.fl <= R(0.5)) {
        // bounce-back solid node: f*_i = f+_opp(i); reversing every link flips the
        // sign of the odd moments (j, q) and keeps the even ones (deviation form too)
        const V2<R> m[4] = {{n.mp[1], n.mp[2]}, {-n.mp[3], -n.mp[5]}, {-n.mp[4], -n.mp[6]}, {n.mp[7], n.mp[8]}};
        R f0;
        V2<R> F[4];
        f_from_m9p<R, kFlowScale<M>>(n.mp[0], m, f0, F);
        store_flow<M>(db, f0, F, PS);
      } else {
        // Eq. 3 at the node's velocity (u = u_b = 0 on walls)
        const R drag = P.drag_lin + P.drag_forch * n.um;
        const V2<R> U = {n.ux, n.uy};
        const V2<R> F = fma2(V2<R>{-drag, -drag}, U, V2<R>{R(0), P.phi * n.Gy});   // (F_x, F_y)
        // blended moments (Eq. 20 in moment space, deviation form); no blend in the
        // bounce-back variant.  Pairs (e, eps), (j_x, j_y), (q_x, q_y), (p_xx, p_xy)
        const R fb = P.solid_scheme ? R(1) : n.fl;
        const R sol = (R(1) - fb) * n.drho;
        const V2<R> FB = {fb, fb};
        V2<R> m12 = fma2(FB, V2<R>{n.mp[1], n.mp[2]}, V2<R>{R(-2) * sol, sol});
        V2<R> m46 = mul2(FB, V2<R>{n.mp[4], n.mp[6]});
        V2<R> m78 = mul2(FB, V2<R>{n.mp[7], n.mp[8]});
        // equilibria (Eq. 18, deviation form) and forcing moments (Eq. 19); the q
        // pair's equilibrium and forcing are the negated j pair's
        const R rho = n.rho, rip = rho * P.inv_phi, drho = n.drho;
        const R q = R(3) * rip * (n.ux * n.ux + n.uy * n.uy);
        const V2<R> me12 = {R(-2) * drho + q, drho - q};
        const V2<R> J = mul2(V2<R>{rho, rho}, U);
        const V2<R> me78 = mul2(V2<R>{rip, rip}, V2<R>{n.ux * n.ux - n.uy * n.uy, n.ux * n.uy});
        const R s1 = R(6) * rip * (n.ux * F.x + n.uy * F.y);
        const V2<R> RF = mul2(V2<R>{rho, rho}, F);
        const V2<R> S78 = mul2(V2<R>{rip, rip}, V2<R>{R(2) * (n.ux * F.x - n.uy * F.y), n.ux * F.y + n.uy * F.x});
        // Eq. 14: the rates of Sec. III C are constants (s_rho = s_j = 1, s_e = s_eps =
        // 1.1, s_q = 1.2); only s_v = s[7] = s[8] depends on the run.  Where s = 1 the
        // result is m^eq + S/2 whatever the blend gave (rho: m^eq = delta_rho, S = 0)
        m12 = fma2(V2<R>{R(0.45), R(0.45)}, V2<R>{s1, -s1},
                   fma2(V2<R>{R(-1.1), R(-1.1)}, sub2(m12, me12), m12));
        const V2<R> m35 = fma2(V2<R>{R(0.5), R(0.5)}, RF, J);
        m46 = fma2(V2<R>{R(-0.4), R(-0.4)}, RF, fma2(V2<R>{R(-1.2), R(-1.2)}, add2(m46, J), m46));
        const R sv = P.s[7], hv = R(1) - R(0.5) * sv;
        m78 = fma2(V2<R>{hv, hv}, S78, fma2(V2<R>{-sv, -sv}, sub2(m78, me78), m78));
        const V2<R> m[4] = {m12, m35, m46, m78};
        R f0;
        V2<R> Fo[4];
        f_from_m9p<R, kFlowScale<M>>(drho, m, f0, Fo);
        store_flow<M>(db, f0, Fo, PS);
      }
    }
}

// PCM and metal collisions and stores of one node (Eqs. 32, 36, 43, 47 with
// the backward difference of Remark III): dTp is the node's exchange history,
// db/dw its element in bulk and wide plane 0 of the next copy; returns the new
// history T_m - T_f.
template <int M, int QT, bool FLOW, bool PH>
__device__ __forceinline__ typename ModeTraits<M>::R thermal_collide(const StepParams<typename ModeTraits<M>::R>& P,
                                                                     NodeState<M, QT, FLOW>& n,
                                                                     typename ModeTraits<M>::R dTp,
                                                                     typename ModeTraits<M>::B* db, float* dw,
                                                                     int PS = kChunk) {
    using R = typename ModeTraits<M>::R;
    // exchange sources, Eqs. 36 and 47 with the backward difference of Remark III
    const R dTn = n.Tm - n.Tf;
    const R Sx = R(1.5) * dTn - R(0.5) * dTp;
    const R S_met = -P.a_m * Sx;
    // metal n_0 after its source (n_0 is conserved by the collision, Eq. 43).  The
    // PCM takes the opposite of what the metal's n_0 actually changed by, scaled
    // by the heat capacities (S_PCM = -(a_f/a_m) S_metal, Eqs. 36, 47), so an
    // exchange that the metal's rounding drops moves no energy into the PCM
    R hm_base;
    if constexpr (kSplit<M>) hm_base = n.th[0].y;
    else hm_base = n.th[0].y - P.eta[0] * (n.th[0].y - n.Tm);
    const R hm = hm_base + S_met;
    const R S_pcm = (hm - hm_base) * P.x_pm;

    // PCM (Eq. 32) and metal (Eq. 43) collisions side by side
    R neg[QT], nem[QT];
    neq_pcm<R, QT>(P, n.H, n.Tf, n.ux, n.uy, neg);
    neq_metal<R, QT>(P, n.Tm, nem);
    V2<R> nr[QT];
#pragma unroll
    for (int k = 1; k < QT; ++k) nr[k] = P.nrate[QT == 5 && k == 2 ? 1 : k];   // D2Q5: j_x, j_y share a rate (App. B)
    if (PH && P.phase_k) {
        // Eq. 9 at the node's liquid fraction -> zeta_alpha (Eq. A19) -> zeta_e (Eq. 53)
        const R za = fast_rcp(R(0.5) + P.ks_c + n.fl * (P.kl_c - P.ks_c));
#pragma unroll
        for (int k = 1; k < QT; ++k) nr[k].x = -(P.zr_a[k] + P.zr_b[k] * za);
    }
#pragma unroll
    for (int k = 1; k < QT; ++k) {
        // both equilibria vanish for k = 4 (D2Q5) and k = 7, 8 (D2Q9)
        const bool zero = QT == 5 ? k == 4 : k >= 7;
        const V2<R> d = zero ? n.th[k] : sub2(n.th[k], V2<R>{neg[k], nem[k]});
        n.th[k] = fma2(nr[k], d, n.th[k]);
    }
    if constexpr (QT == 9) {
        n.th[1] = fma2(V2<R>{R(-2), R(-2)}, V2<R>{S_pcm, S_met}, n.th[1]);
        n.th[2] = add2(n.th[2], V2<R>{S_pcm, S_met});
    } else {
        n.th[3] = fma2(V2<R>{P.varpi, P.varpi}, V2<R>{S_pcm, S_met}, n.th[3]);
    }
    // n_0* = H + S_PCM (n_0 is conserved up to the source, Eq. 32)
    R hi, lo;
    if constexpr (kComp<M>) {
        const FF n0 = ff_add(FF{n.th[0].x, n.Hlo}, S_pcm);
        hi = n0.hi;
        lo = n0.lo;
    } else {
        hi = n.th[0].x + S_pcm;
        lo = R(0);
    }
    store_thermal<M, QT, FLOW>(P, n.th, hi, lo, hm, db, dw, PS);
    return dTn;
}

// Node (x, y)'s element in bulk plane 0 and in wide plane 0 (16-bit modes) of
// the next copy.
template <int M, int QT, bool FLOW>
__device__ __forceinline__ typename ModeTraits<M>::B* next_bulk(const StepParams<typename ModeTraits<M>::R>& P, int x,
                                                                int y) {
    const long long ro = (long long)y * (P.cpr * Chunk<M, QT, FLOW>::bytes);
    return reinterpret_cast<typename ModeTraits<M>::B*>(P.dst + (ro + col_off<M, QT, FLOW>(x)));
}

template <int M, int QT, bool FLOW>
__device__ __forceinline__ float* next_wide(const StepParams<typename ModeTraits<M>::R>& P, int x, int y) {
    if constexpr (kSplit<M>) {
        const long long ro = (long long)y * (P.cpr * Chunk<M, QT, FLOW>::bytes);
        return reinterpret_cast<float*>(P.dst + (ro + col_off<M, QT, FLOW, true>(x)));
    } else {
        return nullptr;
    }
}

// One time step of node (x, y): steps a1-a9 (pull, walls, state, blend,
// velocity, three collisions, store).  PH = true compiles the Eq. 9 variant's
// per-node PCM rates in (taken where P.phase_k is set); PH = false leaves them
// out of the kernel altogether.
template <int M, int QT, bool FLOW, bool PH = false>
__device__ __forceinline__ void step_node(const StepParams<typename ModeTraits<M>::R>& P, int x, int y) {
    using R = typename ModeTraits<M>::R;
    NodeState<M, QT, FLOW> n;
    bool wall;
    node_state<M, QT, FLOW>(P, x, y, n, wall);

    const int o = y * P.pitch + x;                                  // exchange history
    // read before any store: the compiler cannot move it above stores that may
    // alias it, and a load after them adds a memory round trip to the step
    // (256^2 FP32: 2.47 -> 2.37 us per step)
    const R dTp = P.dT[o];
    typename ModeTraits<M>::B* db = next_bulk<M, QT, FLOW>(P, x, y);
    float* dw = next_wide<M, QT, FLOW>(P, x, y);
    flow_collide<M, QT, FLOW>(P, n, db);
    P.dT[o] = thermal_collide<M, QT, FLOW, PH>(P, n, dTp, db, dw);

    // non-finite or runaway state: raise the sticky flag (no trap)
    // (a NaN anywhere fails a comparison; the sum overflows if any term is huge)
    const bool bad = !(fabs(n.H) + fabs(n.Tm) + n.rho < R(1e30)) || !(n.rho > R(0)) ||
                     !(n.ux * n.ux + n.uy * n.uy <= R(0.09));
    if (bad) atomicOr(P.status, STATUS_UNSTABLE);
}

// Blocks of 256 threads each SM must hold, which caps the registers per
// thread: five for the FP32 and 16-bit forms of D2Q5 with flow (48 registers;
// with the packed arithmetic 40 registers and six blocks measured ~1 % slower
// at 256^2 and 2048^2 in FP32); the others take what their registers allow.
template <int M, int QT, bool FLOW>
constexpr int kMinBlocks = (QT == 5 && FLOW) ? (M == MODE_F64 ? 1 : 5) : 1;

// Programmatic dependent launch (sm_90 and later): the step kernels are
// launched as programmatic dependents of the previous step, so their launch
// overlaps its tail.  griddep_wait blocks until the previous grid in the
// stream has completed and its writes are visible (it returns at once when
// this grid was not launched as a programmatic dependent); no thread touches
// the state before it.  The dependents are released when this grid's blocks
// exit (no early trigger: dependents scheduled while this grid still runs took
// its SM resources, 256^2 went from 2.75 to 3.52 us per step; released at exit,
// 2.50).
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// L2 prefetch ahead of the blocks that will run next (node pairs on large
// grids): a block's first thread asks L2, by bulk prefetches
// (cp.async.bulk.prefetch.L2), for the chunk of x in `rows` rows starting at
// y0 and for their exchange history, so that the block launched for those
// rows later finds them in L2 instead of waiting for HBM.  No registers or
// shared memory hold the data; rows past the grid are skipped.
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int M, int QT, bool FLOW>
__device__ __forceinline__ void prefetch_rows(const StepParams<typename ModeTraits<M>::R>& P, int x, int y0, int rows) {
    using R = typename ModeTraits<M>::R;
    constexpr uint32_t cb = Chunk<M, QT, FLOW>::bytes;   // a multiple of 16, as is every chunk's offset
    for (int y = y0; y < y0 + rows && y < P.ny; ++y) {
        l2_prefetch(P.src + ((long long)y * P.cpr + (x >> kChunkShift)) * cb, cb);
        l2_prefetch(P.dT + (long long)y * P.pitch + (x & ~(kChunk - 1)), kChunk * (uint32_t)sizeof(R));
    }
}

// One run: one thread per node, 256 threads per block (128 x 2 by default;
// the batch's map 3 may take other shapes).
template <int M, int QT, bool FLOW, bool PH>
__global__ void __launch_bounds__(256, (kMinBlocks<M, QT, FLOW>)) fused_step(const __grid_constant__ StepParams<typename ModeTraits<M>::R> P) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    griddep_wait();
    step_node<M, QT, FLOW, PH>(P, x, y);
}

// ---------------------------------------------------------------------------
// Two time steps per launch
// ---------------------------------------------------------------------------
// On small grids (state resident in L2) a step costs the launch-to-launch floor
// of a dependent launch plus one warp's dependency chain with its L2 loads,
// more than the issue time of the work itself; on grids whose state exceeds
// L2 a step moves the whole state through HBM.  fused_step2 advances two time
// steps per launch.  A block of kT2W x H threads (one node each, 4 <= H <=
// kT2H) owns an inner tile of (kT2W - 2) x (H - 2) nodes and the one-node ring
// around it:
//   1. every thread advances its node one step from the state in global
//      memory (the ring's nodes belong to neighbouring tiles and are advanced
//      there too), storing the result in shared memory in the storage
//      encoding of a state copy, as a global store would;
//   2. after a barrier, the inner nodes advance a second step with their
//      neighbourhood read from shared memory, and store to the next copy.
// Tile origins are clamped to the grid (the last tile along an axis ends at
// the grid's edge, overlapping its neighbour), so that a wall node's x_f and
// the neighbours of x_f lie in the tile (H >= 4).  Nodes of overlapping tiles
// are computed by both blocks with the same inputs and code, and written with
// the same values.  The history is read from P.dT and written to P.dT_out:
// other blocks still read the previous history of their rings.  Flow runs
// only.  The host picks H per grid (t2_block in the launcher).  Two builds of
// the kernel: HM = kT2H (any H up to 16; one block per SM on the grids that
// take it) and HM = kT2HMany (H = 12 for grids of many tiles per SM, launch
// bounds that leave three FP32 D2Q5 blocks resident: at 52 registers only two
// fit, 2048^2 FP32 104 against 84 us per step; two blocks of the other builds,
// which would spill under the three-block cap).
constexpr int kT2W = 34, kT2H = 16, kT2HMany = 12;

template <int HM, int M, int QT>
constexpr int kT2Blocks = HM == kT2HMany ? (M == MODE_F32 && QT == 5 ? 3 : 2) : 1;

// Dynamic shared memory of a two-step block of up to HM rows, planes
// kT2W * HM elements apart: the bulk planes (storage type), the wide planes
// (FP32) and the history.
template <int M, int QT, int HM>
struct Tile2 {
    using PL = Planes<M, QT, true>;
    static constexpr int n = kT2W * HM;
    static constexpr size_t wide_off = (size_t)PL::bulk * n * sizeof(typename ModeTraits<M>::B);
    static constexpr size_t dT_off = wide_off + (size_t)PL::wide * n * sizeof(float);
    static constexpr size_t bytes = dT_off + (size_t)n * sizeof(typename ModeTraits<M>::R);
    static_assert(wide_off % 16 == 0 && dT_off % 16 == 0, "16-byte aligned parts");
};

// Neighbourhood of the node at tile index i (pull node) in the tile, planes
// PS elements apart.
template <int M, int PS>
struct PullTile {
    const typename ModeTraits<M>::B* b;
    const float* wd;
    int i;
    __device__ __forceinline__ int at(int q) const { return i + (src_row(q) - 1) * kT2W + (src_col(q) - 1); }
    __device__ __forceinline__ typename ModeTraits<M>::R bulk(int q, int plane) const {
        return to_f(b[plane * PS + at(q)]);
    }
    __device__ __forceinline__ float wide(int q, int p) const { return wd[p * PS + at(q)]; }
};

// First node of the ring of tile k along an axis of n nodes with inner width w.
__host__ __device__ __forceinline__ int t2_origin(int k, int w, int n) {
    return (n > w ? min(k * w, n - w) : 0) - 1;
}

// Tiles along an axis of n nodes with inner width w.
__host__ __device__ __forceinline__ int t2_count(int n, int w) { return n > w ? (n + w - 1) / w : 1; }

// Both steps of tile (bx, by) of run P, by a block of kT2W x blockDim.y
// threads (blockDim.y <= HM) with Tile2<M, QT, HM>::bytes of dynamic shared
// memory.
template <int M, int QT, bool PH, int HM>
__device__ __forceinline__ void step2_tile(const StepParams<typename ModeTraits<M>::R>& P, int bx, int by) {
    using R = typename ModeTraits<M>::R;
    using B = typename ModeTraits<M>::B;
    using TL = Tile2<M, QT, HM>;
    extern __shared__ __align__(16) unsigned char t2_smem[];
    B* sb = reinterpret_cast<B*>(t2_smem);
    float* sw = reinterpret_cast<float*>(t2_smem + TL::wide_off);
    R* sdT = reinterpret_cast<R*>(t2_smem + TL::dT_off);
    const int H = blockDim.y;   // blockDim.x == kT2W, H <= HM
    const int lx = threadIdx.x, ly = threadIdx.y, i = ly * kT2W + lx;
    const int X0 = t2_origin(bx, kT2W - 2, P.nx), Y0 = t2_origin(by, H - 2, P.ny);
    // step-1 node: coordinates wrapped on periodic sides, none beyond a walled side
    int x = X0 + lx, y = Y0 + ly;
    bool live = true;
    if (x < 0 || x >= P.nx) {
        if (P.per_x) x = ((x % P.nx) + P.nx) % P.nx;
        else live = false;
    }
    if (y < 0 || y >= P.ny) {
        if (P.per_y) y = ((y % P.ny) + P.ny) % P.ny;
        else live = false;
    }
    griddep_wait();
    if (live) {
        NodeState<M, QT, true> n;
        bool wall;
        node_state<M, QT, true>(P, x, y, n, wall);
        const R dTp = P.dT[y * P.pitch + x];
        flow_collide<M, QT, true>(P, n, sb + i, TL::n);
        sdT[i] = thermal_collide<M, QT, true, PH>(P, n, dTp, sb + i, kSplit<M> ? sw + i : nullptr, TL::n);
        const bool bad = !(fabs(n.H) + fabs(n.Tm) + n.rho < R(1e30)) || !(n.rho > R(0)) ||
                         !(n.ux * n.ux + n.uy * n.uy <= R(0.09));
        if (bad) atomicOr(P.status, STATUS_UNSTABLE);
    }
    __syncthreads();
    // step 2: the inner nodes of the tile that lie in the grid
    const int x2 = X0 + lx, y2 = Y0 + ly;
    if (lx < 1 || lx > kT2W - 2 || ly < 1 || ly > H - 2 || x2 >= P.nx || y2 >= P.ny) return;
    const WallAt wa = wall_at(P, x2, y2);
    const PullTile<M, TL::n> a{sb, sw, i + (wa.ys - y2) * kT2W + (wa.xs - x2)};
    NodeState<M, QT, true> n;
    node_state_from<M, QT, true>(P, a, wa, n);
    flow_collide<M, QT, true>(P, n, next_bulk<M, QT, true>(P, x2, y2));
    P.dT_out[y2 * P.pitch + x2] =
        thermal_collide<M, QT, true, PH>(P, n, sdT[i], next_bulk<M, QT, true>(P, x2, y2), next_wide<M, QT, true>(P, x2, y2));
    const bool bad = !(fabs(n.H) + fabs(n.Tm) + n.rho < R(1e30)) || !(n.rho > R(0)) ||
                     !(n.ux * n.ux + n.uy * n.uy <= R(0.09));
    if (bad) atomicOr(P.status, STATUS_UNSTABLE);
}

template <int M, int QT, bool PH, int HM>
__global__ void __launch_bounds__(kT2W * HM, (kT2Blocks<HM, M, QT>)) fused_step2(const __grid_constant__ StepParams<typename ModeTraits<M>::R> P) {
    step2_tile<M, QT, PH, HM>(P, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Two nodes per thread
// ---------------------------------------------------------------------------
// Large grids of the default configuration (flow, D2Q5 thermal lattices,
// volumetric blend, FP32/FP16/BF16 storage) advance node pairs (x0, x0 + 1),
// x0 even, one pair per thread.  Every FP32 operation of the step is one
// packed instruction for both nodes (lane x: node x0, lane y: node x0 + 1),
// the parameter loads and the index arithmetic serve both nodes, and the pair
// is read and written with one access per plane wherever both elements are
// adjacent (x0 even keeps them inside one chunk, aligned).  The arithmetic is
// that of step_node, operation for operation, except where noted; a pair with
// a wall node (or without a second node) goes through step_node instead.

using W = V2<float>;

__device__ __forceinline__ W wb(float s) { return {s, s}; }
__device__ __forceinline__ W wmin(W a, float b) { return {fminf(a.x, b), fminf(a.y, b)}; }
__device__ __forceinline__ W wmax0(W a) { return {fmaxf(a.x, 0.0f), fmaxf(a.y, 0.0f)}; }
__device__ __forceinline__ W wsat(W a) { return {__saturatef(a.x), __saturatef(a.y)}; }
__device__ __forceinline__ W wrcp(W a) { return {__fdividef(1.0f, a.x), __fdividef(1.0f, a.y)}; }
__device__ __forceinline__ W wsqrt(W a) { return {fast_sqrt(a.x), fast_sqrt(a.y)}; }

// two adjacent elements of a plane (16-bit: one 32-bit access; FP32: 64-bit)
template <int M>
__device__ __forceinline__ W ldw(const char* p) {
    if constexpr (M == MODE_F16) {
        const float2 f = __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
        return {f.x, f.y};
    } else if constexpr (M == MODE_BF16) {
        const float2 f = __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)));
        return {f.x, f.y};
    } else {
        const float2 f = __ldg(reinterpret_cast<const float2*>(p));
        return {f.x, f.y};
    }
}

// stores v; returns the stored values as a reader decodes them
template <int M>
__device__ __forceinline__ W stw(char* p, W v) {
    if constexpr (M == MODE_F16) {
        const __half2 h = __floats2half2_rn(v.x, v.y);
        *reinterpret_cast<__half2*>(p) = h;
        const float2 f = __half22float2(h);
        return {f.x, f.y};
    } else if constexpr (M == MODE_BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
        *reinterpret_cast<__nv_bfloat162*>(p) = h;
        const float2 f = __bfloat1622float2(h);
        return {f.x, f.y};
    } else {
        *reinterpret_cast<float2*>(p) = make_float2(v.x, v.y);
        return v;
    }
}

__device__ __forceinline__ W ldwf(const char* p) {   // two adjacent FP32 elements
    const float2 f = __ldg(reinterpret_cast<const float2*>(p));
    return {f.x, f.y};
}

__device__ __forceinline__ void stwf(char* p, W v) { *reinterpret_cast<float2*>(p) = make_float2(v.x, v.y); }

struct FW {
    W hi, lo;
};

__device__ __forceinline__ FW two_sum(W a, W b) {   // Knuth, lane by lane
    const W s = add2(a, b);
    const W bb = sub2(s, a);
    return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}

__device__ __forceinline__ FW fast_two_sum(W a, W b) {   // Dekker, |a| >= |b|
    const W s = add2(a, b);
    return {s, sub2(b, sub2(s, a))};
}

// as ff_accumulate<5>
__device__ __forceinline__ FW fw_accumulate(FW a, const W* v, float sign) {
    W s = a.hi, c = a.lo;
#pragma unroll
    for (int i = 1; i < 5; ++i) {
        const FW t = two_sum(s, sign == 1.0f ? v[i] : mul2(wb(sign), v[i]));
        s = t.hi;
        c = add2(c, t.lo);
    }
    return fast_two_sum(s, c);
}

__device__ __forceinline__ void enthalpy_state(const StepParams<float>& P, W H, W& T, W& fl) {
    fl = wsat(mul2(sub2(H, wb(P.H_fs)), wb(P.inv_dH)));
    T = add2(fma2(fl, wb(P.dT_sl), wmin(mul2(H, wb(P.inv_c_ps)), P.T_fs)), wmax0(sub2(H, wb(P.H_fl))));
}

__device__ __forceinline__ W pcm_ref(const StepParams<float>& P, W g0) {
    const W a = fma2(wsat(mul2(sub2(g0, wb(P.g0_fs)), wb(P.inv_dg0))), wb(P.cr_dsl), wmin(mul2(g0, wb(P.cr_solid)), P.cr_fs));
    return fma2(wmax0(sub2(g0, wb(P.g0_fl))), wb(P.cr_liquid), a);
}

// D2Q5 moments of one lattice (Eq. B1) and back
__device__ __forceinline__ void m_from_f5w(const W* g, W* n) {
    const W a = add2(g[1], g[3]), b = add2(g[2], g[4]);
    n[1] = sub2(g[1], g[3]);
    n[2] = sub2(g[2], g[4]);
    n[3] = add2(a, b);
    n[4] = sub2(a, b);
    n[0] = add2(g[0], n[3]);
}

__device__ __forceinline__ void f_from_m5w(const W* n, W* g) {
    const W p = mul2(add2(n[3], n[4]), wb(0.25f)), q = mul2(sub2(n[3], n[4]), wb(0.25f));
    g[0] = sub2(n[0], n[3]);
    g[1] = fma2(wb(0.5f), n[1], p);
    g[3] = fma2(wb(-0.5f), n[1], p);
    g[2] = fma2(wb(0.5f), n[2], q);
    g[4] = fma2(wb(-0.5f), n[2], q);
}

// Source of a node pair's pulled neighbourhood in the state copy in global
// memory: plane `plane` in source row r (0: y - 1, 1: y, 2: y + 1) of the pair
// (x0, x0 + 1), of its west neighbours (x0 - 1, x0) and of its east ones
// (x0 + 1, x0 + 2); the wide planes (16-bit modes) of the pair and of the
// nodes x0 - 1, x0 + 2; the pair's exchange history.
template <int M>
struct PairAt {
    using B = typename ModeTraits<M>::B;
    using CH = Chunk<M, 5, true>;
    static constexpr int es = (int)sizeof(B);
    static constexpr int pb = kChunk * es;   // bytes from one bulk plane to the next
    static constexpr int wpl = kChunk * 4;   // bytes from one wide plane to the next
    const char* row[3];
    int c0, cm, cp, w0, wm, wp;
    const float* dT;
    __device__ __forceinline__ PairAt(const StepParams<float>& P, int x0, int y) {
        // neighbour columns of the pair (periodic wrap; no walls reach here)
        const int xm = x0 == 0 ? P.nx - 1 : x0 - 1;   // west of x0
        const int xp = x0 + 2 == P.nx ? 0 : x0 + 2;   // east of x0 + 1
        const int ym = y == 0 ? P.ny - 1 : y - 1;
        const int yp = y == P.ny - 1 ? 0 : y + 1;
        const int rb = P.cpr * CH::bytes;
        row[0] = P.src + (long long)ym * rb;
        row[1] = P.src + (long long)y * rb;
        row[2] = P.src + (long long)yp * rb;
        c0 = col_off<M, 5, true>(x0);
        cm = col_off<M, 5, true>(xm);
        cp = col_off<M, 5, true>(xp);
        w0 = c0 + CH::wide_off + (x0 & (kChunk - 1)) * 2;   // wide element of x0
        wm = cm + CH::wide_off + (xm & (kChunk - 1)) * 2;
        wp = cp + CH::wide_off + (xp & (kChunk - 1)) * 2;
        dT = P.dT + (long long)y * P.pitch + x0;
    }
    __device__ __forceinline__ W own(int r, int q) const { return ldw<M>(row[r] + c0 + q * pb); }
    __device__ __forceinline__ W west(int r, int q) const {
        return W{ldb<M>(reinterpret_cast<const B*>(row[r] + cm + q * pb)),
                 ldb<M>(reinterpret_cast<const B*>(row[r] + c0 + q * pb))};
    }
    __device__ __forceinline__ W east(int r, int q) const {
        return W{ldb<M>(reinterpret_cast<const B*>(row[r] + c0 + q * pb) + 1),
                 ldb<M>(reinterpret_cast<const B*>(row[r] + cp + q * pb))};
    }
    __device__ __forceinline__ W own_wide(int r, int w) const { return ldwf(row[r] + w0 + w * wpl); }
    __device__ __forceinline__ float west_wide(int r, int w) const {
        return __ldg(reinterpret_cast<const float*>(row[r] + wm + w * wpl));
    }
    __device__ __forceinline__ float east_wide(int r, int w) const {
        return __ldg(reinterpret_cast<const float*>(row[r] + wp + w * wpl));
    }
    __device__ __forceinline__ W history() const { return ldwf(reinterpret_cast<const char*>(dT)); }
};

// One time step of the node pair (x0, x0 + 1) of row y, its neighbourhood
// read through the source S (PairAt or a staged copy in shared memory); the
// results go to the next copy and the history array in global memory.
template <int M, bool PH, typename S>
__device__ __forceinline__ void step_pair_from(const StepParams<float>& P, const S& src, int x0, int y) {
    using PL = Planes<M, 5, true>;
    using CH = Chunk<M, 5, true>;
    constexpr int pb = kChunk * (int)sizeof(typename ModeTraits<M>::B);   // plane stride of the next copy
    const int c0 = col_off<M, 5, true>(x0);
    const int rb = P.cpr * CH::bytes;
    auto own = [&](int r, int q) { return src.own(r, q); };
    auto west = [&](int r, int q) { return src.west(r, q); };
    auto east = [&](int r, int q) { return src.east(r, q); };

    // ---- pull (Eq. 15) and flow moments (Eq. 13) ----
    W f[9] = {own(1, 0), west(1, 1), own(0, 2), east(1, 3), own(2, 4), west(0, 5), east(0, 6), east(2, 7), west(2, 8)};
    if constexpr (M == MODE_F16) {
#pragma unroll
        for (int q = 0; q < 9; ++q) f[q] = mul2(f[q], wb(1.0f / 1024.0f));
    }
    W m[9];
    {
        const W A13 = add2(f[1], f[3]), A24 = add2(f[2], f[4]), dx = sub2(f[1], f[3]), dy = sub2(f[2], f[4]);
        const W B57 = add2(f[5], f[7]), B68 = add2(f[6], f[8]), E57 = sub2(f[5], f[7]), E68 = sub2(f[6], f[8]);
        const W s14 = add2(A13, A24), s58 = add2(B57, B68);
        const W ax = sub2(E57, E68), ay = add2(E57, E68);
        m[0] = add2(add2(f[0], s14), s58);
        m[1] = fma2(wb(2.0f), s58, fma2(wb(-1.0f), s14, mul2(wb(-4.0f), f[0])));
        m[2] = fma2(wb(-2.0f), s14, fma2(wb(4.0f), f[0], s58));
        m[3] = add2(dx, ax);
        m[5] = add2(dy, ay);
        m[4] = fma2(wb(-2.0f), dx, ax);
        m[6] = fma2(wb(-2.0f), dy, ay);
        m[7] = sub2(A13, A24);
        m[8] = sub2(B57, B68);
    }

    // ---- thermal pull: PCM g, metal h (Eqs. 33, 44; App. B) ----
    W g[5], h[5];
    W Hlo = wb(0.0f);
    if constexpr (kSplit<M>) {
        const W g0o = src.own_wide(1, 0), h0o = src.own_wide(1, 1);
        // senders' rest populations for movers 1..4 (from x - e_q)
        const W sg[5] = {g0o, W{src.west_wide(1, 0), g0o.x}, src.own_wide(0, 0), W{g0o.y, src.east_wide(1, 0)},
                         src.own_wide(2, 0)};
        const W sh[5] = {h0o, W{src.west_wide(1, 1), h0o.x}, src.own_wide(0, 1), W{h0o.y, src.east_wide(1, 1)},
                         src.own_wide(2, 1)};
        const W dg[5] = {wb(0.0f), west(1, PL::pcm(1)), own(0, PL::pcm(2)), east(1, PL::pcm(3)), own(2, PL::pcm(4))};
        const W dh[5] = {wb(0.0f), west(1, PL::met(1)), own(0, PL::met(2)), east(1, PL::met(3)), own(2, PL::met(4))};
        const float wg = P.wmv[1].x, wk = P.wmv[1].y;   // D2Q5: one weight for all movers (App. B)
        g[0] = g0o;
        h[0] = h0o;
#pragma unroll
        for (int q = 1; q < 5; ++q) {
            g[q] = fma2(wb(wg), pcm_ref(P, sg[q]), dg[q]);
            h[q] = fma2(wb(wk), sh[q], dh[q]);
        }
    } else {
        g[0] = own(1, PL::pcm(0));
        h[0] = own(1, PL::met(0));
        g[1] = west(1, PL::pcm(1)); g[2] = own(0, PL::pcm(2)); g[3] = east(1, PL::pcm(3)); g[4] = own(2, PL::pcm(4));
        h[1] = west(1, PL::met(1)); h[2] = own(0, PL::met(2)); h[3] = east(1, PL::met(3)); h[4] = own(2, PL::met(4));
    }
    W ng[5], nh[5];
    m_from_f5w(g, ng);
    m_from_f5w(h, nh);
    if constexpr (kComp<M>) {   // H = (g_0 hi + g_0 lo) + sum of movers, without rounding loss
        const FW H = fw_accumulate(FW{g[0], own(1, PL::lo)}, g, 1.0f);
        ng[0] = H.hi;
        Hlo = H.lo;
    }

    // ---- macroscopic state (Eqs. 21, 23-25, 37-39, 7) ----
    const W H = ng[0];
    W Tf, fl;
    enthalpy_state(P, H, Tf, fl);
    const W Tm = nh[0];
    const W drho = m[0];
    const W rho = add2(wb(1.0f), drho);
    const W Gy = mul2(mul2(wb(P.gbeta), sub2(Tf, wb(P.T0))), fl);
    W ux, uy, um;
    {
        const W ir = wrcp(rho);
        const W vx = mul2(mul2(fl, m[3]), ir);
        const W vy = fma2(wb(0.5f * P.phi), Gy, mul2(mul2(fl, m[5]), ir));
        const W vm = wsqrt(fma2(vy, vy, mul2(vx, vx)));
        W r = wsqrt(fma2(wb(P.l1), vm, wb(P.l0sq)));
        const W den = wrcp(add2(wb(P.l0), r));   // Eq. 23
        ux = mul2(vx, den);
        uy = mul2(vy, den);
        um = mul2(vm, den);
    }

    // ---- flow collision (Eqs. 3, 14, 18-20) ----
    char* dst = P.dst + (long long)y * rb;
    {
        const W nd = fma2(wb(-P.drag_forch), um, wb(-P.drag_lin));   // -(drag)
        const W Fx = mul2(nd, ux), Fy = fma2(nd, uy, mul2(wb(P.phi), Gy));
        const W sol = mul2(sub2(wb(1.0f), fl), drho);
        W b1 = fma2(fl, m[1], mul2(wb(-2.0f), sol)), b2 = fma2(fl, m[2], sol);
        W b4 = mul2(fl, m[4]), b6 = mul2(fl, m[6]), b7 = mul2(fl, m[7]), b8 = mul2(fl, m[8]);
        const W rip = mul2(rho, wb(P.inv_phi));
        const W uxx = mul2(ux, ux), uyy = mul2(uy, uy), uxy = mul2(ux, uy);
        const W q = mul2(mul2(wb(3.0f), rip), add2(uxx, uyy));
        const W me1 = fma2(wb(-2.0f), drho, q), me2 = sub2(drho, q);
        const W Jx = mul2(rho, ux), Jy = mul2(rho, uy);
        const W me7 = mul2(rip, sub2(uxx, uyy)), me8 = mul2(rip, uxy);
        const W s1 = mul2(mul2(wb(6.0f), rip), fma2(uy, Fy, mul2(ux, Fx)));
        const W RFx = mul2(rho, Fx), RFy = mul2(rho, Fy);
        const W S7 = mul2(rip, mul2(wb(2.0f), sub2(mul2(ux, Fx), mul2(uy, Fy))));
        const W S8 = mul2(rip, fma2(uy, Fx, mul2(ux, Fy)));
        b1 = fma2(wb(0.45f), s1, fma2(wb(-1.1f), sub2(b1, me1), b1));
        b2 = fma2(wb(-0.45f), s1, fma2(wb(-1.1f), sub2(b2, me2), b2));
        const W b3 = fma2(wb(0.5f), RFx, Jx), b5 = fma2(wb(0.5f), RFy, Jy);
        b4 = fma2(wb(-0.4f), RFx, fma2(wb(-1.2f), add2(b4, Jx), b4));
        b6 = fma2(wb(-0.4f), RFy, fma2(wb(-1.2f), add2(b6, Jy), b6));
        const float sv = P.s[7], hv = 1.0f - 0.5f * sv;
        b7 = fma2(wb(hv), S7, fma2(wb(-sv), sub2(b7, me7), b7));
        b8 = fma2(wb(hv), S8, fma2(wb(-sv), sub2(b8, me8), b8));
        // f = M^-1 m* (as f_from_m9p), scaled by the storage scale
        constexpr float sc = (float)kFlowScale<M>;
        const W A = mul2(drho, wb(sc / 9.0f)), Bm = mul2(b1, wb(sc / 36.0f)), C = mul2(b2, wb(sc / 36.0f));
        const W DX = mul2(b3, wb(sc / 6.0f)), QX = mul2(b4, wb(sc / 12.0f));
        const W DY = mul2(b5, wb(sc / 6.0f)), QY = mul2(b6, wb(sc / 12.0f));
        const W Pm = mul2(b7, wb(sc * 0.25f)), Sm = mul2(b8, wb(sc * 0.25f));
        const W f0 = fma2(wb(4.0f), C, fma2(wb(-4.0f), Bm, A));
        const W bb1 = fma2(wb(-2.0f), C, sub2(A, Bm));
        const W bb5 = add2(fma2(wb(2.0f), Bm, A), C);
        const W Tx = fma2(wb(-2.0f), QX, DX), Ty = fma2(wb(-2.0f), QY, DY);
        const W X = add2(DX, QX), Y = add2(DY, QY);
        const W bp = add2(bb1, Pm), bm = sub2(bb1, Pm);
        const W G5 = add2(bb5, Sm), G6 = sub2(bb5, Sm), H5 = add2(X, Y), H6 = sub2(Y, X);
        const W fo[9] = {f0, add2(bp, Tx), add2(bm, Ty), sub2(bp, Tx), sub2(bm, Ty),
                         add2(G5, H5), add2(G6, H6), sub2(G5, H5), sub2(G6, H6)};
#pragma unroll
        for (int k = 0; k < 9; ++k) stw<M>(dst + c0 + k * pb, fo[k]);
    }

    // ---- exchange sources (Eqs. 36, 47, Remark III) ----
    // (the history is read here, after the flow stores: read with the other
    // loads it stays live through the step and costs FP16 a spill, 72.9
    // against 70.2 us per step at 2048^2)
    float* dTp_ptr = P.dT + (long long)y * P.pitch + x0;
    const W dTn = sub2(Tm, Tf);
    const W dTp = src.history();
    const W Sx = fma2(wb(1.5f), dTn, mul2(wb(-0.5f), dTp));
    const W S_met = mul2(wb(-P.a_m), Sx);
    W hm_base;
    if constexpr (kSplit<M>) hm_base = nh[0];
    else hm_base = fma2(wb(-P.eta[0]), sub2(nh[0], Tm), nh[0]);
    const W hm = add2(hm_base, S_met);
    const W S_pcm = mul2(sub2(hm, hm_base), wb(P.x_pm));

    // ---- PCM (Eq. 32) and metal (Eq. 43) collisions ----
    {
        const W t = mul2(Tf, wb(P.inv_phi));
        const W ne1 = mul2(t, ux), ne2 = mul2(t, uy), ne3 = mul2(wb(P.vcf), Tf);
        W nz[5];
        if (PH && P.phase_k) {   // Eq. 9 -> zeta_alpha (Eq. A19) -> zeta_e (Eq. 53)
            const W za = wrcp(add2(wb(0.5f + P.ks_c), mul2(fl, wb(P.kl_c - P.ks_c))));
#pragma unroll
            for (int k = 1; k < 5; ++k) nz[k] = mul2(wb(-1.0f), fma2(wb(P.zr_b[k]), za, wb(P.zr_a[k])));
        } else {
            nz[1] = nz[2] = wb(P.nrate[1].x);
            nz[3] = wb(P.nrate[3].x);
            nz[4] = wb(P.nrate[4].x);
        }
        ng[1] = fma2(nz[1], sub2(ng[1], ne1), ng[1]);
        ng[2] = fma2(nz[2], sub2(ng[2], ne2), ng[2]);
        ng[3] = fma2(nz[3], sub2(ng[3], ne3), ng[3]);
        ng[4] = fma2(nz[4], ng[4], ng[4]);
        const float ne_j = P.nrate[1].y;
        nh[1] = fma2(wb(ne_j), nh[1], nh[1]);
        nh[2] = fma2(wb(ne_j), nh[2], nh[2]);
        nh[3] = fma2(wb(P.nrate[3].y), sub2(nh[3], mul2(wb(P.vcm), Tm)), nh[3]);
        nh[4] = fma2(wb(P.nrate[4].y), nh[4], nh[4]);
        ng[3] = fma2(wb(P.varpi), S_pcm, ng[3]);
        nh[3] = fma2(wb(P.varpi), S_met, nh[3]);
    }
    // n_0* = H + S_PCM (Eq. 32), metal n_0* = hm
    W n0hi, n0lo = wb(0.0f);
    if constexpr (kComp<M>) {
        const FW s = two_sum(ng[0], S_pcm);
        const FW n0 = fast_two_sum(s.hi, add2(s.lo, Hlo));
        n0hi = n0.hi;
        n0lo = n0.lo;
    } else {
        n0hi = add2(ng[0], S_pcm);
    }

    // ---- thermal store: movers, then the rest populations as remainders ----
    W vg[5], vh[5];
    ng[0] = n0hi;
    nh[0] = hm;
    f_from_m5w(ng, vg);
    f_from_m5w(nh, vh);
    if constexpr (kSplit<M>) {
        // as store_thermal: deviations from the provisional rest population's
        // reference, then the rest population that closes the balance
        const W ref = pcm_ref(P, vg[0]);
        const float nwg = P.nwmv[1].x, nwk = P.nwmv[1].y;
        W sdg, sdh;
#pragma unroll
        for (int k = 1; k < 5; ++k) {
            const W dgk = stw<M>(dst + c0 + PL::pcm(k) * pb, fma2(wb(nwg), ref, vg[k]));
            const W dhk = stw<M>(dst + c0 + PL::met(k) * pb, fma2(wb(nwk), vh[0], vh[k]));
            sdg = k == 1 ? dgk : add2(sdg, dgk);
            sdh = k == 1 ? dhk : add2(sdh, dhk);
        }
        const W Yg = sub2(n0hi, sdg), Yh = sub2(hm, sdh);
        W T, f_;
        enthalpy_state(P, Yg, T, f_);
        const int w0 = c0 + CH::wide_off + (x0 & (kChunk - 1)) * 2;
        stwf(dst + w0, fma2(wb(-P.om_cf), T, Yg));
        stwf(dst + w0 + kChunk * 4, mul2(Yh, wb(P.rest_m)));
    } else {
#pragma unroll
        for (int k = 1; k < 5; ++k) {
            stw<M>(dst + c0 + PL::pcm(k) * pb, vg[k]);
            stw<M>(dst + c0 + PL::met(k) * pb, vh[k]);
        }
        const W smh = add2(add2(add2(vh[1], vh[2]), vh[3]), vh[4]);
        stw<M>(dst + c0 + PL::met(0) * pb, sub2(hm, smh));
        if constexpr (kComp<M>) {   // the PCM rest population as a float-float pair
            const FW r = fw_accumulate(FW{n0hi, n0lo}, vg, -1.0f);
            stw<M>(dst + c0 + PL::pcm(0) * pb, r.hi);
            stw<M>(dst + c0 + PL::lo * pb, r.lo);
        } else {
            const W smg = add2(add2(add2(vg[1], vg[2]), vg[3]), vg[4]);
            stw<M>(dst + c0 + PL::pcm(0) * pb, sub2(n0hi, smg));
        }
    }
    stwf(reinterpret_cast<char*>(dTp_ptr), dTn);

    // non-finite or runaway state: raise the sticky flag (no trap)
    const W a = add2(add2(W{fabsf(H.x), fabsf(H.y)}, W{fabsf(Tm.x), fabsf(Tm.y)}), rho);
    const W u2 = fma2(uy, uy, mul2(ux, ux));
    const bool bad = !(a.x < 1e30f) || !(a.y < 1e30f) || !(rho.x > 0.0f) || !(rho.y > 0.0f) ||
                     !(u2.x <= 0.09f) || !(u2.y <= 0.09f);
    if (bad) atomicOr(P.status, STATUS_UNSTABLE);
}

template <int M, bool PH>
__device__ __forceinline__ void step_pair(const StepParams<float>& P, int x0, int y) {
    const PairAt<M> src(P, x0, y);
    step_pair_from<M, PH>(P, src, x0, y);
}

// Node pairs of the default configuration: a block of 32 x 4 threads covers
// 64 x 4 nodes; the first of a chunk's two blocks prefetches its rows (2048^2
// FP16 61.09 against 61.22 us per step when both do).  A pair with a wall node or without a second node (or a run
// of the bounce-back variant) takes step_node.  Seven blocks per SM cap the
// registers at 72 (measured best: 80 registers leave too few warps to hide
// the memory latency, 64 spill).
template <int M, bool PH>
__global__ void __launch_bounds__(128, 7) fused_step_pair(const __grid_constant__ StepParams<float> P) {
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x0 >= P.nx || y >= P.ny) return;
    griddep_wait();
    if (P.prefetch_rows > 0 && threadIdx.x == 0 && threadIdx.y == 0 && (x0 & (kChunk - 1)) == 0)
        prefetch_rows<M, 5, true>(P, x0, y + P.prefetch_rows, blockDim.y);   // the chunk's first block
    const bool single = P.solid_scheme || x0 + 1 >= P.nx || (!P.per_x && (x0 == 0 || x0 + 1 == P.nx - 1)) ||
                        (!P.per_y && (y == 0 || y == P.ny - 1));
    if (single) {
        step_node<M, 5, true, PH>(P, x0, y);
        if (x0 + 1 < P.nx) step_node<M, 5, true, PH>(P, x0 + 1, y);
        return;
    }
    step_pair<M, PH>(P, x0, y);
}

// Many small runs in one launch per step, each run on the code of the
// single-run kernel (map 4 of a batch).  The parameter blocks of up to
// kGroupRuns runs travel in the kernel's own parameter space (the constant
// bank, up to 32 KB), with the prefix sums of the runs' block counts; block b
// finds its run by a binary search over them (uniform across the block) and
// takes block b - first_block[run] of that run's tiles: w x (128 / w) nodes,
// one node per thread (fused_step's arithmetic), w = 32 << tile[run] chosen so
// that the run's width leaves the fewest threads idle.  With all small runs in
// one grid the device sees one large launch instead of many small ones, each
// bound by the latency of a few warps.
template <typename R>
constexpr int kGroupRuns = (32000 - 16) / (int)(sizeof(StepParams<R>) + 2 * sizeof(int));

template <typename R>
struct GroupParams {
    int nruns;
    int first_block[kGroupRuns<R> + 1];
    int tile[kGroupRuns<R>];
    StepParams<R> run[kGroupRuns<R>];
};

template <int M, int QT, bool FLOW, bool PH>
__global__ void __launch_bounds__(128, 2 * kMinBlocks<M, QT, FLOW>) group_step(
    const __grid_constant__ GroupParams<typename ModeTraits<M>::R> G) {
    using R = typename ModeTraits<M>::R;
    const int b = blockIdx.x;
    int lo = 0, hi = G.nruns - 1;   // the last run whose first block is <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (G.first_block[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const StepParams<R>& P = G.run[lo];
    const int lb = b - G.first_block[lo];
    const int lw = 5 + G.tile[lo];   // log2 of the tile width
    const int t = (int)threadIdx.x;
    const int gx = (P.nx + (1 << lw) - 1) >> lw;
    const int x = (lb % gx) * (1 << lw) + (t & ((1 << lw) - 1));
    const int y = (lb / gx) * (128 >> lw) + (t >> lw);
    if (x >= P.nx || y >= P.ny) return;
    griddep_wait();
    step_node<M, QT, FLOW, PH>(P, x, y);
}

// Batch map 5: the grouped launch of the two-step form.  Run k owns blocks
// first_block[k] .. first_block[k + 1] - 1, one per two-step tile (blocks of
// kT2W x kT2HMany threads, inner tiles of (kT2W - 2) x (kT2HMany - 2) nodes,
// row-major over the run's tiles); each block advances its tile two steps as
// fused_step2 does, with its run's parameter block.
template <int M, int QT, bool PH>
__global__ void __launch_bounds__(kT2W * kT2HMany, (kT2Blocks<kT2HMany, M, QT>)) group_step2(
    const __grid_constant__ GroupParams<typename ModeTraits<M>::R> G) {
    using R = typename ModeTraits<M>::R;
    const int b = blockIdx.x;
    int lo = 0, hi = G.nruns - 1;   // the last run whose first block is <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (G.first_block[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const StepParams<R>& P = G.run[lo];
    const int lb = b - G.first_block[lo];
    const int gx = t2_count(P.nx, kT2W - 2);
    step2_tile<M, QT, PH, kT2HMany>(P, lb % gx, lb / gx);
}

// Many runs in one launch.  A tile is w x (256 / w) nodes of one run (w a
// power of two, 32..256); thread t of a block takes node (x0 + t mod w,
// y0 + t div w).  Each run has two parameter blocks in global memory, one per
// ping-pong direction ([run][2]); a run whose current copy differs from the
// batch's parity carries flip = 1 in its tiles.  A block copies the block of
// its current run into shared memory when the run changes.  Map: chunk > 0
// gives block b the tiles [b chunk, (b+1) chunk), chunk = 0 strides over the
// tiles by the grid size.
struct Tile {
    int run, x0, y0, log2w_flip;   // log2 w in bits 0-7, flip in bit 8
};

template <int M, int QT, bool FLOW, bool PH>
__global__ void __launch_bounds__(256) batch_step(const StepParams<typename ModeTraits<M>::R>* __restrict__ runs,
                                                  const Tile* __restrict__ tiles, int ntiles, int chunk, int parity) {
    using R = typename ModeTraits<M>::R;
    __shared__ StepParams<R> P;
    static_assert(sizeof(StepParams<R>) % 4 == 0, "parameter block copied as words");
    int cached = -1;
    const int t0 = chunk > 0 ? blockIdx.x * chunk : blockIdx.x;
    const int t1 = chunk > 0 ? min(ntiles, t0 + chunk) : ntiles;
    const int dt = chunk > 0 ? 1 : gridDim.x;
    for (int t = t0; t < t1; t += dt) {
        const Tile tl = tiles[t];
        if (tl.run != cached) {   // uniform across the block
            __syncthreads();
            const int dir = parity ^ ((tl.log2w_flip >> 8) & 1);
            const int* src = reinterpret_cast<const int*>(runs + 2 * tl.run + dir);
            int* dst = reinterpret_cast<int*>(&P);
            for (int i = threadIdx.x; i < (int)(sizeof(StepParams<R>) / 4); i += blockDim.x) dst[i] = __ldg(src + i);
            __syncthreads();
            cached = tl.run;
        }
        const int lg = tl.log2w_flip & 0xff;
        const int x = tl.x0 + (threadIdx.x & ((1 << lg) - 1));
        const int y = tl.y0 + (threadIdx.x >> lg);
        if (x < P.nx && y < P.ny) step_node<M, QT, FLOW, PH>(P, x, y);
    }
}

// Fields at the current time level (LBM_FIELD_* order).
template <typename R>
struct FieldOut {
    R* dst[7];
    int mask;
    int ld;   // row stride of the outputs (elements)
};

template <int M, int QT, bool FLOW>
__global__ void __launch_bounds__(256) fields_kernel(const __grid_constant__ StepParams<typename ModeTraits<M>::R> P,
                                                     const __grid_constant__ FieldOut<typename ModeTraits<M>::R> out) {
    using R = typename ModeTraits<M>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    NodeState<M, QT, FLOW> n;
    bool wall;
    node_state<M, QT, FLOW>(P, x, y, n, wall);
    const long long o = (long long)y * out.ld + x;
    const R v[7] = {n.Tf, n.Tm, n.fl, n.ux, n.uy, n.rho, n.H};   // H: high part
#pragma unroll
    for (int i = 0; i < 7; ++i)
        if (out.mask & (1 << i)) out.dst[i][o] = v[i];
}

// Diagnostics: per-block FP64 partial sums of f_l, enthalpy, mass and the
// left-wall heat flux, written to scratch[block][4] in a fixed order.
struct DiagConst {
    double phi, rho_l, rho_m, c_pm, k_f, k_s, k_m;   // k_f: liquid PCM conductivity, k_s: solid (Eq. 9)
    int left_wall;  // 1 when x = 0 is a wall (Nusselt number defined)
};

template <int M, int QT, bool FLOW>
__global__ void __launch_bounds__(256) diag_partial(const __grid_constant__ StepParams<typename ModeTraits<M>::R> P,
                                                    const __grid_constant__ DiagConst C,
                                                    double* __restrict__ scratch) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (x < P.nx && y < P.ny) {
        NodeState<M, QT, FLOW> n;
        bool wall;
        node_state<M, QT, FLOW>(P, x, y, n, wall);
        v[0] = (double)n.fl;
        v[1] = C.phi * C.rho_l * ((double)n.H + (double)n.Hlo) +
               (1.0 - C.phi) * C.rho_m * C.c_pm * ((double)n.Tm + (double)n.Elo);
        v[2] = 1.0 + (double)n.drho;
        if (x == 0 && C.left_wall && P.nx >= 3) {
            NodeState<M, QT, FLOW> n1, n2;
            bool w1, w2;
            node_state<M, QT, FLOW>(P, 1, y, n1, w1);
            node_state<M, QT, FLOW>(P, 2, y, n2, w2);
            const double gf = 0.5 * (3.0 * (double)n.Tf - 4.0 * (double)n1.Tf + (double)n2.Tf);
            const double gm = 0.5 * (3.0 * (double)n.Tm - 4.0 * (double)n1.Tm + (double)n2.Tm);
            // PCM conductivity of the wall node's own liquid fraction (Eq. 9)
            const double kw = C.k_s == C.k_f ? C.k_f : (double)n.fl * C.k_f + (1.0 - (double)n.fl) * C.k_s;
            v[3] = C.phi * kw * gf + (1.0 - C.phi) * C.k_m * gm;
        }
    }
    __shared__ double red[4][32];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        double a = v[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
        if (lane == 0) red[i][warp] = a;
    }
    __syncthreads();
    if (tid < 4) {
        double a = 0.0;
        for (int w = 0; w < nwarps; ++w) a += red[tid][w];
        scratch[(long long)(blockIdx.y * gridDim.x + blockIdx.x) * 4 + tid] = a;
    }
}

// Sums the partials in a fixed order (one block of 256 threads).
__global__ void diag_finalize(const double* __restrict__ scratch, int nblocks, double* __restrict__ out);

}  // namespace lbmk
