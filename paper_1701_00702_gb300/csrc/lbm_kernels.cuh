// Device code of the fused three-lattice time step (Liu, He & Li, arXiv
// 1701.00702, Sec. III).  One thread owns one node; the whole step is one
// pass over HBM: 9 + 2*Q_T populations and the exchange history are read
// once (pull streaming, Eqs. 15, 33, 44) and written once.
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
//     with error-free additions (Knuth's TwoSum, Dekker's Fast2Sum), and the
//     post-collision rest population is the remainder g_0* = n_0* - sum_{i>=1}
//     g_i* of the rounded moving populations, so that streaming and collision
//     conserve the enthalpy to ~2^-48 instead of accumulating FP32 rounding
//     in the isothermal mushy zone, where nothing damps it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmk {

// Per-run constants, passed by value (__grid_constant__).
template <typename R>
struct StepParams {
    const R* src;        // [planes][ny][pitch]: 9 flow planes (if flow), Q_T PCM, Q_T metal
    R* dst;
    R* dT;               // [ny][pitch] exchange history T_m - T_f of the previous step
    unsigned int* status;
    int nx, ny, pitch;
    long long plane;     // ny * pitch
    int per_x, per_y;
    int wall_kind[4];
    R wall_T[4], wall_H[4], wall_H_lo[4];
    // flow (Eqs. 3, 7, 16, 25)
    R phi, inv_phi, drag_lin, drag_forch, gbeta, T0, l0, l0sq, l1;
    R s[9];
    // thermal (Eqs. 38-39, 34, 45, App. B)
    R H_fs, H_fl, inv_dH, mush_slope, T_fs, T_fl, inv_c_ps, inv_c_pl;
    R c_pl, c_fref, c_mref, c_pm, inv_c_pm, varpi;
    R zeta[9], eta[9];
    R a_f, a_m;          // h_v/(phi rho_l), h_v/((1 - phi) rho_m)
};

enum : unsigned int { STATUS_UNSTABLE = 1u };

// FP32 storage keeps the PCM rest population as a float-float pair.
template <typename R>
constexpr bool kComp = sizeof(R) == 4;

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

__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const FF s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, a.lo), b.lo));
}

__device__ __forceinline__ FF ff_neg(FF a) { return {-a.hi, -a.lo}; }

// Exact-ish sum of the moving populations v[1..Q-1].
template <int Q>
__device__ __forceinline__ FF ff_sum_movers(const float* v) {
    FF acc = {v[1], 0.0f};
#pragma unroll
    for (int i = 2; i < Q; ++i) acc = ff_add(acc, v[i]);
    return acc;
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

template <typename R>
__device__ __forceinline__ void f_from_m9(const R* m, R* f) {
    const R A = m[0] * R(1.0 / 9.0), B = m[1] * R(1.0 / 36.0), C = m[2] * R(1.0 / 36.0);
    const R DX = m[3] * R(1.0 / 6.0), QX = m[4] * R(1.0 / 12.0);
    const R DY = m[5] * R(1.0 / 6.0), QY = m[6] * R(1.0 / 12.0);
    const R P = m[7] * R(0.25), S = m[8] * R(0.25);
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

template <typename R>
__device__ __forceinline__ void m_from_f5(const R* g, R* n) {
    n[0] = g[0] + g[1] + g[2] + g[3] + g[4];
    n[1] = g[1] - g[3];
    n[2] = g[2] - g[4];
    n[3] = g[1] + g[2] + g[3] + g[4];
    n[4] = g[1] - g[2] + g[3] - g[4];
}

template <typename R>
__device__ __forceinline__ void f_from_m5(const R* n, R* g) {
    const R p = (n[3] + n[4]) * R(0.25), q = (n[3] - n[4]) * R(0.25);
    g[0] = n[0] - n[3];
    g[1] = R(0.5) * n[1] + p;
    g[3] = R(-0.5) * n[1] + p;
    g[2] = R(0.5) * n[2] + q;
    g[4] = R(-0.5) * n[2] + q;
}

template <typename R, int Q>
__device__ __forceinline__ void fwd(const R* v, R* m) {
    if constexpr (Q == 9) m_from_f9(v, m); else m_from_f5(v, m);
}

template <typename R, int Q>
__device__ __forceinline__ void inv(const R* m, R* v) {
    if constexpr (Q == 9) f_from_m9(m, v); else f_from_m5(m, v);
}

// ---------------------------------------------------------------------------
// Equilibrium moments
// ---------------------------------------------------------------------------

// Eq. 18 (alpha_1 = 1, alpha_2 = -3) minus the rest moments r = (1, -2, 1, 0, ..., 0);
// rho = 1 + drho.
template <typename R>
__device__ __forceinline__ void meq_flow_dev(const StepParams<R>& P, R rho, R drho, R ux, R uy, R* me) {
    const R ip = P.inv_phi;
    const R q = R(3) * rho * (ux * ux + uy * uy) * ip;
    me[0] = drho;
    me[1] = R(-2) * drho + q;
    me[2] = drho - q;
    me[3] = rho * ux;
    me[4] = -rho * ux;
    me[5] = rho * uy;
    me[6] = -rho * uy;
    me[7] = rho * (ux * ux - uy * uy) * ip;
    me[8] = rho * ux * uy * ip;
}

// Eq. 34 (D2Q9) / Eq. B2 (D2Q5)
template <typename R, int Q>
__device__ __forceinline__ void neq_pcm(const StepParams<R>& P, R H, R T, R ux, R uy, R* ne) {
    const R jx = P.c_pl * T * ux * P.inv_phi, jy = P.c_pl * T * uy * P.inv_phi;
    if constexpr (Q == 9) {
        ne[0] = H;
        ne[1] = R(-4) * H + R(2) * P.c_fref * T;
        ne[2] = R(4) * H - R(3) * P.c_fref * T;
        ne[3] = jx; ne[4] = -jx; ne[5] = jy; ne[6] = -jy;
        ne[7] = R(0); ne[8] = R(0);
    } else {
        ne[0] = H; ne[1] = jx; ne[2] = jy; ne[3] = P.varpi * P.c_fref * T; ne[4] = R(0);
    }
}

// Eq. 45 (D2Q9) / Eq. B4 (D2Q5)
template <typename R, int Q>
__device__ __forceinline__ void neq_metal(const StepParams<R>& P, R Tm, R* ne) {
    if constexpr (Q == 9) {
        const R e = P.c_pm * Tm;
        ne[0] = e;
        ne[1] = R(-4) * e + R(2) * P.c_mref * Tm;
        ne[2] = R(4) * e - R(3) * P.c_mref * Tm;
#pragma unroll
        for (int k = 3; k < 9; ++k) ne[k] = R(0);
    } else {
        ne[0] = P.c_pm * Tm; ne[1] = R(0); ne[2] = R(0); ne[3] = P.varpi * P.c_mref * Tm; ne[4] = R(0);
    }
}

// Eqs. 38-39
template <typename R>
__device__ __forceinline__ void enthalpy_state(const StepParams<R>& P, R H, R& T, R& fl) {
    if (H <= P.H_fs) {
        T = H * P.inv_c_ps;
        fl = R(0);
    } else if (H < P.H_fl) {
        const R d = H - P.H_fs;
        T = P.T_fs + d * P.mush_slope;
        fl = d * P.inv_dH;
    } else {
        T = P.T_fl + (H - P.H_fl) * P.inv_c_pl;
        fl = R(1);
    }
}

// ---------------------------------------------------------------------------
// Node state
// ---------------------------------------------------------------------------

template <typename R, int QT, bool FLOW>
struct NodeState {
    R mp[FLOW ? 9 : 1];  // moments of f+ minus r (after the wall rule)
    R ng[QT], nh[QT];    // moments of g and h (after the wall rule); ng[0] = H (high part)
    R Hlo;               // low part of H (float-float bookkeeping; 0 with FP64 storage)
    R H, Tf, fl, Tm, rho, drho, ux, uy, Gy;
};

// Pull streaming around node (xs, ys): the population along e_i comes from
// xs - e_i.  The index wrap is also correct for interior nodes of a walled
// direction, which never reach the edge.
template <typename R, int QT, bool FLOW>
__device__ __forceinline__ void pull_moments(const StepParams<R>& P, int xs, int ys,
                                             NodeState<R, QT, FLOW>& n) {
    const int xm = xs == 0 ? P.nx - 1 : xs - 1;
    const int xp = xs == P.nx - 1 ? 0 : xs + 1;
    const int ym = ys == 0 ? P.ny - 1 : ys - 1;
    const int yp = ys == P.ny - 1 ? 0 : ys + 1;
    const long long r0 = (long long)ys * P.pitch, rm = (long long)ym * P.pitch, rp = (long long)yp * P.pitch;
    const R* __restrict__ s = P.src;
    const long long pl = P.plane;
    int base = 0;
    if constexpr (FLOW) {
        R f[9];
        f[0] = __ldg(s + 0 * pl + r0 + xs);
        f[1] = __ldg(s + 1 * pl + r0 + xm);
        f[2] = __ldg(s + 2 * pl + rm + xs);
        f[3] = __ldg(s + 3 * pl + r0 + xp);
        f[4] = __ldg(s + 4 * pl + rp + xs);
        f[5] = __ldg(s + 5 * pl + rm + xm);
        f[6] = __ldg(s + 6 * pl + rm + xp);
        f[7] = __ldg(s + 7 * pl + rp + xp);
        f[8] = __ldg(s + 8 * pl + rp + xm);
        m_from_f9(f, n.mp);
        base = 9;
    }
    R g[QT], h[QT];
    const R* sg = s + (long long)base * pl;
    const R* sh = s + (long long)(base + QT) * pl;
    g[0] = __ldg(sg + 0 * pl + r0 + xs);
    g[1] = __ldg(sg + 1 * pl + r0 + xm);
    g[2] = __ldg(sg + 2 * pl + rm + xs);
    g[3] = __ldg(sg + 3 * pl + r0 + xp);
    g[4] = __ldg(sg + 4 * pl + rp + xs);
    h[0] = __ldg(sh + 0 * pl + r0 + xs);
    h[1] = __ldg(sh + 1 * pl + r0 + xm);
    h[2] = __ldg(sh + 2 * pl + rm + xs);
    h[3] = __ldg(sh + 3 * pl + r0 + xp);
    h[4] = __ldg(sh + 4 * pl + rp + xs);
    if constexpr (QT == 9) {
        g[5] = __ldg(sg + 5 * pl + rm + xm);
        g[6] = __ldg(sg + 6 * pl + rm + xp);
        g[7] = __ldg(sg + 7 * pl + rp + xp);
        g[8] = __ldg(sg + 8 * pl + rp + xm);
        h[5] = __ldg(sh + 5 * pl + rm + xm);
        h[6] = __ldg(sh + 6 * pl + rm + xp);
        h[7] = __ldg(sh + 7 * pl + rp + xp);
        h[8] = __ldg(sh + 8 * pl + rp + xm);
    }
    fwd<R, QT>(g, n.ng);
    fwd<R, QT>(h, n.nh);
    if constexpr (kComp<R>) {
        // H = (g_0 hi + g_0 lo) + sum of movers, without rounding loss
        const float lo = __ldg(s + (long long)(base + 2 * QT) * pl + r0 + xs);
        const FF H = ff_add(FF{g[0], lo}, ff_sum_movers<QT>(g));
        n.ng[0] = H.hi;
        n.Hlo = H.lo;
    } else {
        n.Hlo = R(0);
    }
}

// Macroscopic state from the moments (Eqs. 21, 23-25, 37-39, 48, 7).
template <typename R, int QT, bool FLOW>
__device__ __forceinline__ void macro(const StepParams<R>& P, NodeState<R, QT, FLOW>& n, bool wall) {
    n.H = n.ng[0];
    enthalpy_state(P, n.H, n.Tf, n.fl);
    n.Tm = n.nh[0] * P.inv_c_pm;
    if constexpr (FLOW) {
        n.drho = n.mp[0];
        n.rho = R(1) + n.drho;
        n.Gy = P.gbeta * (n.Tf - P.T0) * n.fl;
        if (wall) {
            n.ux = R(0);
            n.uy = R(0);
        } else {
            // Eq. 24 with sum_i e_i f_i = f_l sum_i e_i f+_i (the equilibrium at rest carries no momentum)
            const R ir = R(1) / n.rho;
            const R vx = n.fl * n.mp[3] * ir;
            const R vy = n.fl * n.mp[5] * ir + R(0.5) * P.phi * n.Gy;
            const R vm = sqrt(vx * vx + vy * vy);
            const R den = R(1) / (P.l0 + sqrt(P.l0sq + P.l1 * vm));   // Eq. 23
            n.ux = vx * den;
            n.uy = vy * den;
        }
    } else {
        n.drho = R(0);
        n.rho = R(1);
        n.ux = R(0);
        n.uy = R(0);
        n.Gy = R(0);
    }
}

// Full state of node (x, y): interior nodes pull at themselves; wall nodes pull
// at x_f = x_b + inward normal and apply Eq. 52 in moment space.
template <typename R, int QT, bool FLOW>
__device__ __forceinline__ void node_state(const StepParams<R>& P, int x, int y,
                                           NodeState<R, QT, FLOW>& n, bool& wall) {
    const bool wx = !P.per_x && (x == 0 || x == P.nx - 1);
    const bool wy = !P.per_y && (y == 0 || y == P.ny - 1);
    wall = wx || wy;
    const int xs = wx ? (x == 0 ? 1 : P.nx - 2) : x;
    const int ys = wy ? (y == 0 ? 1 : P.ny - 2) : y;
    pull_moments<R, QT, FLOW>(P, xs, ys, n);
    macro<R, QT, FLOW>(P, n, false);
    if (!wall) return;

    const int side = wx ? (x == 0 ? 0 : 1) : (y == 0 ? 2 : 3);
    R Tb, Hb, Tmb;
    if (P.wall_kind[side] == 0) {
        Tb = P.wall_T[side];
        Tmb = Tb;
        Hb = P.wall_H[side];
    } else {
        Tb = n.Tf;
        Hb = n.H;
        Tmb = n.Tm;
    }
    R a[QT], b[QT];
    if constexpr (FLOW) {
        // m^eq(rho_f, 0) - m^eq(rho_f, u_f), written out so that the rho r parts cancel exactly
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
    neq_pcm<R, QT>(P, Hb, Tb, R(0), R(0), a);
    neq_pcm<R, QT>(P, n.H, n.Tf, n.ux, n.uy, b);
#pragma unroll
    for (int k = 1; k < QT; ++k) n.ng[k] += a[k] - b[k];
    if (P.wall_kind[side] == 0) {   // n_0 = H_b exactly (adiabatic: n_0 = H(x_f), unchanged)
        n.ng[0] = P.wall_H[side];
        n.Hlo = P.wall_H_lo[side];
    }
    neq_metal<R, QT>(P, Tmb, a);
    neq_metal<R, QT>(P, n.Tm, b);
#pragma unroll
    for (int k = 0; k < QT; ++k) n.nh[k] += a[k] - b[k];
    macro<R, QT, FLOW>(P, n, true);
}

// ---------------------------------------------------------------------------
// The fused step
// ---------------------------------------------------------------------------

template <typename R, int QT, bool FLOW>
__global__ void __launch_bounds__(256) fused_step(const __grid_constant__ StepParams<R> P) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;

    NodeState<R, QT, FLOW> n;
    bool wall;
    node_state<R, QT, FLOW>(P, x, y, n, wall);

    const long long o = (long long)y * P.pitch + x;
    R* __restrict__ d = P.dst;
    const long long pl = P.plane;
    int base = 0;

    if constexpr (FLOW) {
        // Eq. 3 at the node's velocity (u = u_b = 0 on walls)
        const R um = sqrt(n.ux * n.ux + n.uy * n.uy);
        const R drag = P.drag_lin + P.drag_forch * um;
        const R Fx = -drag * n.ux;
        const R Fy = -drag * n.uy + P.phi * n.Gy;
        // blended moments (Eq. 20 in moment space, deviation form)
        R m[9];
        const R sol = (R(1) - n.fl) * n.drho;
#pragma unroll
        for (int k = 0; k < 9; ++k) m[k] = n.fl * n.mp[k];
        m[0] += sol;
        m[1] -= R(2) * sol;
        m[2] += sol;
        R me[9];
        meq_flow_dev(P, n.rho, n.drho, n.ux, n.uy, me);
        const R ip = P.inv_phi, rho = n.rho;
        const R uF = n.ux * Fx + n.uy * Fy;
        const R S[9] = {R(0), rho * R(6) * uF * ip, -rho * R(6) * uF * ip, rho * Fx, -rho * Fx,
                        rho * Fy, -rho * Fy, rho * R(2) * (n.ux * Fx - n.uy * Fy) * ip,
                        rho * (n.ux * Fy + n.uy * Fx) * ip};
#pragma unroll
        for (int k = 0; k < 9; ++k) m[k] = m[k] - P.s[k] * (m[k] - me[k]) + (R(1) - R(0.5) * P.s[k]) * S[k];
        R f[9];
        f_from_m9(m, f);
#pragma unroll
        for (int k = 0; k < 9; ++k) d[k * pl + o] = f[k];
        base = 9;
    }

    // exchange sources, Eqs. 36 and 47 with the backward difference of Remark III
    const R dTn = n.Tm - n.Tf;
    const R dTp = P.dT[o];
    const R Sx = R(1.5) * dTn - R(0.5) * dTp;
    const R S_pcm = P.a_f * Sx;
    const R S_met = -P.a_m * Sx;

    {
        R ne[QT];
        neq_pcm<R, QT>(P, n.H, n.Tf, n.ux, n.uy, ne);
#pragma unroll
        for (int k = 1; k < QT; ++k) n.ng[k] -= P.zeta[k] * (n.ng[k] - ne[k]);
        if constexpr (QT == 9) {
            n.ng[1] -= R(2) * S_pcm; n.ng[2] += S_pcm;
        } else {
            n.ng[3] += P.varpi * S_pcm;
        }
        // n_0* = H + S_PCM (n_0 is conserved up to the source, Eq. 32)
        R g[QT];
        if constexpr (kComp<R>) {
            const FF n0 = ff_add(FF{n.ng[0], n.Hlo}, S_pcm);
            n.ng[0] = n0.hi;
            inv<R, QT>(n.ng, g);
            const FF g0 = ff_add(n0, ff_neg(ff_sum_movers<QT>(g)));   // rest = exact remainder
            d[(base + 0) * pl + o] = g0.hi;
            d[(long long)(base + 2 * QT) * pl + o] = g0.lo;
        } else {
            n.ng[0] += S_pcm;
            inv<R, QT>(n.ng, g);
            R sm = g[1];
#pragma unroll
            for (int k = 2; k < QT; ++k) sm += g[k];
            d[(base + 0) * pl + o] = n.ng[0] - sm;
        }
#pragma unroll
        for (int k = 1; k < QT; ++k) d[(base + k) * pl + o] = g[k];
    }
    {
        R ne[QT];
        neq_metal<R, QT>(P, n.Tm, ne);
#pragma unroll
        for (int k = 0; k < QT; ++k) n.nh[k] -= P.eta[k] * (n.nh[k] - ne[k]);
        if constexpr (QT == 9) {
            n.nh[0] += S_met; n.nh[1] -= R(2) * S_met; n.nh[2] += S_met;
        } else {
            n.nh[0] += S_met; n.nh[3] += P.varpi * S_met;
        }
        R h[QT];
        inv<R, QT>(n.nh, h);
#pragma unroll
        for (int k = 0; k < QT; ++k) d[(base + QT + k) * pl + o] = h[k];
    }
    P.dT[o] = dTn;

    // non-finite or runaway state: raise the sticky flag (no trap)
    const bool bad = !(fabs(n.H) < R(1e30)) || !(n.rho > R(0) && n.rho < R(1e30)) ||
                     !(n.ux * n.ux + n.uy * n.uy <= R(0.09)) || !(fabs(n.Tm) < R(1e30));
    if (bad) atomicOr(P.status, STATUS_UNSTABLE);
}

// Fields at the current time level (LBM_FIELD_* order).
template <typename R>
struct FieldOut {
    R* dst[7];
    int mask;
    int ld;   // row stride of the outputs (elements)
};

template <typename R, int QT, bool FLOW>
__global__ void __launch_bounds__(256) fields_kernel(const __grid_constant__ StepParams<R> P,
                                                     const __grid_constant__ FieldOut<R> out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    NodeState<R, QT, FLOW> n;
    bool wall;
    node_state<R, QT, FLOW>(P, x, y, n, wall);
    const long long o = (long long)y * out.ld + x;
    const R v[7] = {n.Tf, n.Tm, n.fl, n.ux, n.uy, n.rho, n.H};
#pragma unroll
    for (int i = 0; i < 7; ++i)
        if (out.mask & (1 << i)) out.dst[i][o] = v[i];
}

// Diagnostics: per-block FP64 partial sums of f_l, enthalpy, mass and the
// left-wall heat flux, written to scratch[block][4] in a fixed order.
struct DiagConst {
    double phi, rho_l, rho_m, c_pm, k_f, k_m;
    int left_wall;  // 1 when x = 0 is a wall (Nusselt number defined)
};

template <typename R, int QT, bool FLOW>
__global__ void __launch_bounds__(256) diag_partial(const __grid_constant__ StepParams<R> P,
                                                    const __grid_constant__ DiagConst C,
                                                    double* __restrict__ scratch) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (x < P.nx && y < P.ny) {
        NodeState<R, QT, FLOW> n;
        bool wall;
        node_state<R, QT, FLOW>(P, x, y, n, wall);
        v[0] = (double)n.fl;
        v[1] = C.phi * C.rho_l * ((double)n.H + (double)n.Hlo) + (1.0 - C.phi) * C.rho_m * C.c_pm * (double)n.Tm;
        v[2] = 1.0 + (double)n.drho;
        if (x == 0 && C.left_wall && P.nx >= 3) {
            NodeState<R, QT, FLOW> n1, n2;
            bool w1, w2;
            node_state<R, QT, FLOW>(P, 1, y, n1, w1);
            node_state<R, QT, FLOW>(P, 2, y, n2, w2);
            const double gf = 0.5 * (3.0 * (double)n.Tf - 4.0 * (double)n1.Tf + (double)n2.Tf);
            const double gm = 0.5 * (3.0 * (double)n.Tm - 4.0 * (double)n1.Tm + (double)n2.Tm);
            v[3] = C.phi * C.k_f * gf + (1.0 - C.phi) * C.k_m * gm;
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
