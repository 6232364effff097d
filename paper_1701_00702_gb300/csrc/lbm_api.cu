// Host runtime behind the C ABI of include/lbm.h: parameter map and checks,
// device state, graph-replayed stepping, fields, diagnostics, state I/O.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <new>
#include <type_traits>
#include <utility>
#include <vector>

#include "lbm.h"
#include "lbm_launch.cuh"

namespace lbmk {
LBMK_EXTERN(MODE_F64)
LBMK_EXTERN(MODE_F32)
LBMK_EXTERN(MODE_F16)
LBMK_EXTERN(MODE_BF16)
}  // namespace lbmk

static_assert(LBM_STEP_FORM_AUTO == lbmk::FORM_AUTO && LBM_STEP_FORM_SINGLE == lbmk::FORM_SINGLE &&
                  LBM_STEP_FORM_PAIRS == lbmk::FORM_PAIRS && LBM_STEP_FORM_TWO_STEPS == lbmk::FORM_TWO_STEPS,
              "step form values");

namespace {

constexpr int kGraphSteps = 64;          // steps per captured graph (even: the graph starts and ends on buffer 0)
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool finite(double v) { return std::isfinite(v); }

// Inverse of Eq. 38: T <= T_fs is solid, T >= T_fl (above T_fs) liquid, else mushy.
double enthalpy_of_T(const lbm_params& p, double L_a, double T) {
    const double c_ps = p.cps_over_cpl, c_pl = 1.0;
    const double Hfs = c_ps * p.T_solidus, Hfl = c_pl * p.T_liquidus + L_a;
    if (T <= p.T_solidus) return c_ps * T;
    if (T >= p.T_liquidus) return Hfl + c_pl * (T - p.T_liquidus);
    return Hfs + (T - p.T_solidus) / (p.T_liquidus - p.T_solidus) * (Hfl - Hfs);
}

int derive_impl(const lbm_params* pp, lbm_derived* out) {
    if (!pp) return LBM_ERR_ARG;
    const lbm_params& p = *pp;
    if (p.nx < 1 || p.ny < 1 || p.nx > 65536 || p.ny > 65536) return LBM_ERR_ARG;
    if ((int64_t)p.nx * p.ny > (int64_t(1) << 30)) return LBM_ERR_ARG;
    if ((p.periodic_x != 0 && p.periodic_x != 1) || (p.periodic_y != 0 && p.periodic_y != 1)) return LBM_ERR_ARG;
    if (!p.periodic_x && p.nx < 3) return LBM_ERR_ARG;
    if (!p.periodic_y && p.ny < 3) return LBM_ERR_ARG;
    if (p.thermal_q != 5 && p.thermal_q != 9) return LBM_ERR_ARG;
    if (p.precision != LBM_F64 && p.precision != LBM_F32 && p.precision != LBM_F16 && p.precision != LBM_BF16)
        return LBM_ERR_ARG;
    if (p.flow != 0 && p.flow != 1) return LBM_ERR_ARG;
    for (int s = 0; s < 4; ++s) {
        if (p.wall_kind[s] != LBM_WALL_DIRICHLET && p.wall_kind[s] != LBM_WALL_ADIABATIC) return LBM_ERR_ARG;
        if (!finite(p.wall_T[s])) return LBM_ERR_ARG;
    }
    const double vals[] = {p.porosity, p.Ste, p.cond_ratio, p.Nu_i, p.sigma_hat, p.dp_over_L, p.k_f,
                           p.cfref_over_cpl, p.cmref_over_cpm, p.T_hot, p.T_cold, p.T_init, p.T_ref0,
                           p.T_solidus, p.T_liquidus, p.L_char, p.ks_over_kl, p.cps_over_cpl};
    for (double v : vals)
        if (!finite(v)) return LBM_ERR_ARG;
    if (!(p.porosity > 0.0 && p.porosity < 1.0)) return LBM_ERR_ARG;
    if (!(p.Ste > 0.0) || !(p.k_f > 0.0) || !(p.L_char > 0.0) || !(p.dp_over_L > 0.0)) return LBM_ERR_ARG;
    if (!(p.cfref_over_cpl > 0.0) || !(p.cmref_over_cpm > 0.0) || !(p.sigma_hat > 0.0)) return LBM_ERR_ARG;
    if (!(p.cond_ratio > 0.0) || !(p.Nu_i >= 0.0)) return LBM_ERR_ARG;
    if (!(p.ks_over_kl > 0.0) || !(p.cps_over_cpl > 0.0)) return LBM_ERR_ARG;
    if (!(p.T_liquidus >= p.T_solidus) || p.T_hot == p.T_cold) return LBM_ERR_ARG;
    if (p.thermal_q == 5 && !(p.varpi > 0.0 && p.varpi < 1.0)) return LBM_ERR_ARG;
    if ((p.thermal_collision != 0 && p.thermal_collision != 1) || (p.solid_scheme != 0 && p.solid_scheme != 1))
        return LBM_ERR_ARG;
    if (!finite(p.zeta_e) || p.zeta_e < 0.0) return LBM_ERR_ARG;
    if (p.flow) {
        const double fv[] = {p.Ra, p.Pr, p.Da, p.J, p.F_phi};
        for (double v : fv)
            if (!finite(v)) return LBM_ERR_ARG;
        if (!(p.Pr > 0.0) || !(p.Da > 0.0) || !(p.J > 0.0) || !(p.Ra >= 0.0)) return LBM_ERR_ARG;
    }

    // Eq. 54 with delta_x = delta_t = c = 1, rho_l = 1, c_pl = c_pm = 1; c_ps and
    // k_s from the Eq. 9 ratios (1 and 1 in Sec. IV).
    lbm_derived d;
    std::memset(&d, 0, sizeof d);
    const double rho_l = 1.0, c_pl = 1.0, c_pm = 1.0;
    const double L = p.L_char, dT = p.T_hot - p.T_cold, phi = p.porosity;
    d.alpha_f = p.k_f / (rho_l * c_pl);
    d.nu_f = p.flow ? p.Pr * d.alpha_f : 0.0;
    d.nu_e = p.flow ? p.J * d.nu_f : 0.0;
    d.gbeta = p.flow ? p.Ra * d.nu_f * d.alpha_f / (dT * L * L * L) : 0.0;
    d.K = p.flow ? p.Da * L * L : 0.0;
    d.k_m = p.cond_ratio * p.k_f;
    d.rho_m = p.sigma_hat * rho_l * c_pl / c_pm;
    d.L_a = c_pl * dT / p.Ste;
    if (!(d.L_a > 0.0)) return LBM_ERR_ARG;   // needs T_hot > T_cold
    d.d_p = p.dp_over_L * L;
    d.h_v = p.Nu_i * p.k_f / (d.d_p * d.d_p);
    d.c_fref = p.cfref_over_cpl * c_pl;
    d.c_mref = p.cmref_over_cpm * c_pm;
    d.alpha_fref = p.k_f / (rho_l * d.c_fref);
    d.alpha_mref = d.k_m / (d.rho_m * d.c_mref);
    const double cs2 = 1.0 / 3.0;
    d.csT2 = p.thermal_q == 9 ? cs2 : 0.5 * p.varpi;
    d.c_ps = p.cps_over_cpl * c_pl;
    d.k_s = p.ks_over_kl * p.k_f;
    d.F_phi = p.F_phi >= 0.0 ? p.F_phi : 1.75 / std::sqrt(150.0 * phi * phi * phi);   // Eq. 4 (Ergun)
    d.H_fs = d.c_ps * p.T_solidus;
    d.H_fl = c_pl * p.T_liquidus + d.L_a;
    d.exchange_rate = d.h_v * (1.0 / (phi * rho_l) + 1.0 / ((1.0 - phi) * d.rho_m));

    const double s_v = p.flow ? 1.0 / (0.5 + d.nu_e / cs2) : 1.0;
    const double za = 1.0 / (0.5 + d.alpha_fref / d.csT2);
    const double za_s = 1.0 / (0.5 + d.k_s / (rho_l * d.c_fref) / d.csT2);   // Eq. A19 with k_s
    d.zeta_a_solid = za_s;
    const double ea = 1.0 / (0.5 + d.alpha_mref / d.csT2);
    const double ze = p.zeta_e > 0.0 ? p.zeta_e : 2.0 - za;   // Eq. 53, or Sec. V D's explicit value
    const double s9[9] = {1.0, 1.1, 1.1, 1.0, 1.2, 1.0, 1.2, s_v, s_v};
    std::memcpy(d.s, s9, sizeof s9);
    if (p.thermal_q == 9) {
        const double z9[9] = {1.0, ze, ze, za, za, za, za, 1.2, 1.2};
        const double e9[9] = {1.0, 1.1, 1.1, ea, ea, ea, ea, 1.2, 1.2};
        std::memcpy(d.zeta, z9, sizeof z9);
        std::memcpy(d.eta, e9, sizeof e9);
    } else {
        const double z5[5] = {1.0, za, za, ze, 1.2};   // App. B: Theta = diag(z0, za, za, ze, z_eps)
        const double e5[5] = {1.0, ea, ea, 1.1, 1.2};
        std::memcpy(d.zeta, z5, sizeof z5);
        std::memcpy(d.eta, e5, sizeof e5);
    }
    if (p.thermal_collision == 1)                      // Sec. V A: BGK thermal lattices
        for (int k = 0; k < p.thermal_q; ++k) {
            d.zeta[k] = za;
            d.eta[k] = ea;
        }
    if (p.flow) {
        d.l0 = 0.5 * (1.0 + phi * 0.5 * d.nu_f / d.K);  // Eq. 25
        d.l1 = phi * 0.5 * d.F_phi / std::sqrt(d.K);
    }
    for (int s = 0; s < 4; ++s) d.H_wall[s] = enthalpy_of_T(p, d.L_a, p.wall_T[s]);

    // stability ranges
    auto in02 = [](double r) { return r > 0.0 && r < 2.0; };
    if (p.flow && (!in02(s_v) || !(d.l0 > 0.0))) return LBM_ERR_STABILITY;
    if (!in02(za) || !in02(ea) || !in02(ze)) return LBM_ERR_STABILITY;
    if (!in02(za_s) || !(p.zeta_e > 0.0 || in02(2.0 - za_s))) return LBM_ERR_STABILITY;
    const double cap = p.thermal_q == 9 ? 9.0 / 5.0 : 1.0 / p.varpi;   // Remark I (and its D2Q5 analogue)
    if (!(d.c_fref < cap * std::min(c_pl, d.c_ps)) || !(d.c_mref < cap * c_pm)) return LBM_ERR_STABILITY;
    if (!(d.exchange_rate < 1.0)) return LBM_ERR_STABILITY;
    if (out) *out = d;
    return LBM_OK;
}

struct Layout {
    int pitch, nplanes, nwide;
    int cpr;          // chunks of lbmk::kChunk nodes per row
    size_t chunk_bytes;   // one chunk: every plane of kChunk nodes
    size_t elem;      // bytes of one bulk element (8, 4 or 2)
    size_t relem;     // bytes of one arithmetic element (8 or 4): history, fields, state I/O
    size_t copy_bytes, dT_bytes, off_buf1, off_dT, off_status, off_scratch, off_out, total;
    int nblocks;
};

bool split_mode(int precision) { return precision == LBM_F16 || precision == LBM_BF16; }

Layout layout_of(const lbm_params& p) {
    Layout L;
    const bool split = split_mode(p.precision);
    L.elem = p.precision == LBM_F64 ? 8 : (split ? 2 : 4);
    L.relem = p.precision == LBM_F64 ? 8 : 4;
    // bulk planes: flow (9, deviations), PCM and metal populations; FP32 adds the low
    // part of the PCM rest population; 16-bit modes keep both rest populations in
    // two FP32 "wide" planes.  A copy is [ny][cpr] chunks, each [plane][kChunk]
    // (the bulk planes, then the wide planes); the history is [ny][pitch].
    const int fb = p.flow ? 9 : 0;
    L.nplanes = split ? fb + 2 * (p.thermal_q - 1) : fb + 2 * p.thermal_q + (p.precision == LBM_F32 ? 1 : 0);
    L.nwide = split ? 2 : 0;
    L.cpr = (p.nx + lbmk::kChunk - 1) / lbmk::kChunk;
    L.pitch = L.cpr * lbmk::kChunk;
    L.chunk_bytes = (size_t)lbmk::kChunk * (L.nplanes * L.elem + L.nwide * 4);
    L.copy_bytes = align_up((size_t)L.cpr * p.ny * L.chunk_bytes);
    L.dT_bytes = align_up((size_t)L.pitch * p.ny * L.relem);
    L.nblocks = lbmk::diag_blocks(p.nx, p.ny);
    L.off_buf1 = L.copy_bytes;
    L.off_dT = 2 * L.copy_bytes;
    L.off_status = L.off_dT + L.dT_bytes;
    L.off_scratch = L.off_status + kAlign;
    L.off_out = L.off_scratch + align_up((size_t)L.nblocks * 4 * sizeof(double));
    L.total = L.off_out + kAlign;
    return L;
}

}  // namespace

struct lbm_handle {
    lbm_params p;
    lbm_derived d;
    Layout L;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    lbm_alloc_fn alloc = nullptr;
    lbm_free_fn release = nullptr;
    void* ctx = nullptr;
    char* base = nullptr;
    void* buf[2] = {nullptr, nullptr};
    void* dT = nullptr;
    void* dT2 = nullptr;   // second history array of the two-step form (allocated on first use)
    int t2h = 0;              // its block height (chosen with dT2)
    unsigned int* status = nullptr;
    double* scratch = nullptr;
    double* diag_out = nullptr;
    int cur = 0;
    int64_t steps = 0;
    int sticky = LBM_OK;
    int form = 0;   // step form (LBM_STEP_FORM_*)
    cudaGraphExec_t graph = nullptr;
};

namespace {

void* dev_alloc(lbm_handle* h, size_t bytes) {
    if (h->alloc) return h->alloc(bytes, h->ctx);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, h->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(lbm_handle* h, void* p) {
    if (!p) return;
    if (h->release) h->release(p, h->ctx);
    else cudaFreeAsync(p, h->stream);
}

// 1 when the run takes the Eq. 9 per-node PCM rates (k_s != k_l).
int phase_k_of(const lbm_handle* h) { return h->d.k_s != h->p.k_f ? 1 : 0; }

template <typename R>
lbmk::StepParams<R> make_params(const lbm_handle* h, int from) {
    const lbm_params& p = h->p;
    const lbm_derived& d = h->d;
    lbmk::StepParams<R> P;
    std::memset(&P, 0, sizeof P);
    P.src = static_cast<const char*>(h->buf[from]);
    P.dst = static_cast<char*>(h->buf[1 - from]);
    P.cpr = h->L.cpr;
    P.dT = static_cast<R*>(h->dT);
    P.dT_out = static_cast<R*>(h->dT2);
    P.status = h->status;
    P.nx = p.nx;
    P.ny = p.ny;
    P.pitch = h->L.pitch;
    P.per_x = p.periodic_x;
    P.per_y = p.periodic_y;
    P.solid_scheme = p.solid_scheme;
    P.prefetch_rows = lbmk::prefetch_rows_for(p.precision, p.thermal_q, p.flow, p.solid_scheme,
                                              (long long)p.nx * p.ny, h->form);
    for (int s = 0; s < 4; ++s) {
        P.wall_kind[s] = p.wall_kind[s];
        P.wall_T[s] = (R)p.wall_T[s];
        P.wall_T_lo[s] = (R)(p.wall_T[s] - (double)(R)p.wall_T[s]);
        P.wall_H[s] = (R)d.H_wall[s];
        P.wall_H_lo[s] = (R)(d.H_wall[s] - (double)(R)d.H_wall[s]);
    }
    // FP16 keeps flow deviations (|f_i - w_i| < 1 while |u| < 0.3) in its normal range
    P.fscale = p.precision == LBM_F16 ? (R)1024.0 : (R)1.0;
    P.finv = (R)1.0 / P.fscale;
    {   // references of the 16-bit moving thermal populations (equilibria of Eqs. 40, 49, B3, B5 at u = 0)
        const int Q = p.thermal_q;
        const double om = Q == 9 ? 5.0 / 9.0 : p.varpi;
        const double w9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
        for (int k = 0; k < 9; ++k) P.w_move[k] = (R)(Q == 9 ? w9[k] : 0.25 * p.varpi);
        const double g0fs = d.H_fs - om * d.c_fref * p.T_solidus, g0fl = d.H_fl - om * d.c_fref * p.T_liquidus;
        P.g0_fs = (R)g0fs;
        P.g0_fl = (R)g0fl;
        P.cr_solid = (R)(d.c_fref / (d.c_ps - om * d.c_fref));
        P.cr_liquid = (R)(d.c_fref / (1.0 - om * d.c_fref));
        P.cr_fs = (R)(d.c_fref * p.T_solidus);
        P.cr_dsl = (R)(d.c_fref * (p.T_liquidus - p.T_solidus));
        P.inv_dg0 = (R)(1.0 / (g0fl - g0fs));
        const double kappa = d.c_mref / (1.0 - om * d.c_mref);
        P.kappa_m = (R)kappa;
        for (int k = 0; k < 9; ++k) P.wk_move[k] = (R)((Q == 9 ? w9[k] : 0.25 * p.varpi) * kappa);
        for (int k = 0; k < 9; ++k) {
            P.wmv[k] = {P.w_move[k], P.wk_move[k]};
            P.nwmv[k] = {-P.w_move[k], -P.wk_move[k]};
        }
        P.om_cf = (R)(om * d.c_fref);
        P.rest_m = (R)(1.0 - om * d.c_mref);
    }
    const double phi = p.porosity;
    P.phi = (R)phi;
    P.inv_phi = (R)(1.0 / phi);
    if (p.flow) {
        P.drag_lin = (R)(phi * d.nu_f / d.K);
        P.drag_forch = (R)(phi * d.F_phi / std::sqrt(d.K));
        P.gbeta = (R)d.gbeta;
        P.T0 = (R)p.T_ref0;
        P.l0 = (R)d.l0;
        P.l0sq = (R)(d.l0 * d.l0);
        P.l1 = (R)d.l1;
    }
    for (int k = 0; k < 9; ++k) {
        P.s[k] = (R)d.s[k];
        P.eta[k] = (R)d.eta[k];
        P.nrate[k] = {-(R)d.zeta[k], -(R)d.eta[k]};
    }
    P.H_fs = (R)d.H_fs;
    P.H_fl = (R)d.H_fl;
    P.inv_dH = (R)(1.0 / (d.H_fl - d.H_fs));
    P.dT_sl = (R)(p.T_liquidus - p.T_solidus);
    P.T_fs = (R)p.T_solidus;
    P.T_fl = (R)p.T_liquidus;
    P.inv_c_ps = (R)(1.0 / d.c_ps);
    P.c_fref = (R)d.c_fref;
    P.c_mref = (R)d.c_mref;
    P.varpi = (R)p.varpi;
    P.vcf = (R)(p.varpi * d.c_fref);
    P.vcm = (R)(p.varpi * d.c_mref);
    // Eq. 9 variant: per-node zeta_alpha = 1/(1/2 + k_f(f_l)/(rho_l c_fref c_sT^2)) (Eq. A19);
    // rate k of the PCM lattice is zr_a[k] + zr_b[k] zeta_alpha (fixed, zeta_alpha, or 2 - zeta_alpha)
    P.phase_k = phase_k_of(h);
    P.kl_c = (R)(p.k_f / (d.c_fref * d.csT2));
    P.ks_c = (R)(d.k_s / (d.c_fref * d.csT2));
    {
        const int Q = p.thermal_q, e_role = p.zeta_e > 0.0 ? 0 : 2;
        int role[9] = {0, 1, 1, e_role, 0, 0, 0, 0, 0};
        if (Q == 9) {
            const int r9[9] = {0, e_role, e_role, 1, 1, 1, 1, 0, 0};
            std::memcpy(role, r9, sizeof r9);
        }
        if (p.thermal_collision == 1)
            for (int k = 0; k < Q; ++k) role[k] = 1;
        for (int k = 0; k < 9; ++k) {
            P.zr_a[k] = role[k] == 0 ? (R)d.zeta[k] : (role[k] == 1 ? (R)0.0 : (R)2.0);
            P.zr_b[k] = role[k] == 0 ? (R)0.0 : (role[k] == 1 ? (R)1.0 : (R)-1.0);
        }
    }
    P.a_m = (R)(d.h_v / ((1.0 - phi) * d.rho_m));
    P.x_pm = (R)(-(1.0 - phi) * d.rho_m / (phi * 1.0));
    return P;
}

template <int M>
cudaError_t launch_convert_mode(lbm_handle* h, const lbmk::DenseState<typename lbmk::ModeTraits<M>::R>& D,
                                int to_dense) {
    using R = typename lbmk::ModeTraits<M>::R;
    return lbmk::launch_convert<M>(make_params<R>(h, h->cur), D, to_dense, h->p.thermal_q, h->p.flow, h->stream);
}

int cuda_fail(lbm_handle* h) {
    cudaGetLastError();
    if (h) h->sticky = LBM_ERR_CUDA;
    return LBM_ERR_CUDA;
}

// One step of run h from copy `from` with its step form (form < 0) or the given one.
cudaError_t enqueue_one(lbm_handle* h, int from, cudaStream_t s, int form = -1) {
    const int q = h->p.thermal_q, fl = h->p.flow, fm = form < 0 ? h->form : form;
    switch (h->p.precision) {
        case LBM_F64: return lbmk::launch_step<lbmk::MODE_F64>(make_params<double>(h, from), q, fl, fm, s);
        case LBM_F32: return lbmk::launch_step<lbmk::MODE_F32>(make_params<float>(h, from), q, fl, fm, s);
        case LBM_F16: return lbmk::launch_step<lbmk::MODE_F16>(make_params<float>(h, from), q, fl, fm, s);
        default: return lbmk::launch_step<lbmk::MODE_BF16>(make_params<float>(h, from), q, fl, fm, s);
    }
}

// Two steps from copy `from` into the other copy.  The history goes from h->dT
// to h->dT2 in the first launch of a pair and back in the second (back = 1),
// so that it is in h->dT after every even number of launches.
cudaError_t enqueue_two(lbm_handle* h, int from, int back, cudaStream_t s) {
    const int q = h->p.thermal_q;
    auto run = [&](auto P, auto tag) {
        if (back) std::swap(P.dT, P.dT_out);
        return lbmk::launch_step2<decltype(tag)::value>(P, q, h->t2h, s);
    };
    switch (h->p.precision) {
        case LBM_F32: return run(make_params<float>(h, from), std::integral_constant<int, lbmk::MODE_F32>{});
        case LBM_F16: return run(make_params<float>(h, from), std::integral_constant<int, lbmk::MODE_F16>{});
        case LBM_BF16: return run(make_params<float>(h, from), std::integral_constant<int, lbmk::MODE_BF16>{});
        default: return cudaErrorInvalidConfiguration;
    }
}

bool two_steps(const lbm_handle* h) {
    return lbmk::two_steps_for(h->p.precision, h->p.thermal_q, h->p.flow, (long long)h->p.nx * h->p.ny, h->form);
}

// The second history array and the block height of the two-step form, on
// first use (the SM count of the current device).
int ensure_dT2(lbm_handle* h) {
    if (h->dT2) return LBM_OK;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cuda_fail(h);
    h->t2h = lbmk::t2_block(h->p.nx, h->p.ny, nsm);
    h->dT2 = dev_alloc(h, h->L.dT_bytes);
    return h->dT2 ? LBM_OK : LBM_ERR_OOM;
}

// kGraphSteps steps from copy 0 back to copy 0: single steps, or kGraphSteps / 2
// two-step launches (an even number, so the history ends in h->dT).
int build_graph(lbm_handle* h) {
    if (h->graph) return LBM_OK;
    if (!h->cap && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) return cuda_fail(h);
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return cuda_fail(h);
    cudaError_t e = cudaSuccess;
    if (two_steps(h)) {
        for (int i = 0; i < kGraphSteps / 2 && e == cudaSuccess; ++i) e = enqueue_two(h, i & 1, i & 1, h->cap);
    } else {
        for (int i = 0; i < kGraphSteps && e == cudaSuccess; ++i) e = enqueue_one(h, i & 1, h->cap);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(h);
    }
    cudaError_t e3 = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) {
        h->graph = nullptr;
        return cuda_fail(h);
    }
    return LBM_OK;
}

int sync_and_check(lbm_handle* h) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h);
    unsigned int st = 0;
    if (cudaMemcpy(&st, h->status, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess) return cuda_fail(h);
    if (st & lbmk::STATUS_UNSTABLE) h->sticky = LBM_ERR_UNSTABLE;
    return h->sticky;
}

void init_values(const lbm_handle* h, lbmk::InitVals& V) {
    const lbm_params& p = h->p;
    const lbm_derived& d = h->d;
    const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    const double T = p.T_init, H = enthalpy_of_T(p, d.L_a, T);
    for (int i = 0; i < 9; ++i) V.f[i] = 0.0;            // f^eq(1, 0) - w_i = 0 (Eq. 27, deviation storage)
    const int Q = p.thermal_q;
    // g^eq(H, T, 0): Eq. 40 / B3; h^eq(T): Eq. 49 / B5 (c_pl = c_pm = 1)
    const double gw0 = Q == 9 ? 5.0 / 9.0 : p.varpi;
    V.g[0] = H - gw0 * d.c_fref * T;
    V.h[0] = T - gw0 * d.c_mref * T;
    for (int i = 1; i < Q; ++i) {
        const double wi = Q == 9 ? w[i] : 0.25 * p.varpi;
        V.g[i] = wi * d.c_fref * T;
        V.h[i] = wi * d.c_mref * T;
    }
    V.g0_lo = V.g[0] - (double)(float)V.g[0];            // low part of g_0 (FP32 storage)
}

cudaError_t enqueue_init(lbm_handle* h) {
    lbmk::InitVals V;
    std::memset(&V, 0, sizeof V);
    init_values(h, V);
    const int q = h->p.thermal_q, fl = h->p.flow;
    cudaStream_t s = h->stream;
    switch (h->p.precision) {
        case LBM_F64: return lbmk::launch_init<lbmk::MODE_F64>(make_params<double>(h, 0), V, q, fl, s);
        case LBM_F32: return lbmk::launch_init<lbmk::MODE_F32>(make_params<float>(h, 0), V, q, fl, s);
        case LBM_F16: return lbmk::launch_init<lbmk::MODE_F16>(make_params<float>(h, 0), V, q, fl, s);
        default: return lbmk::launch_init<lbmk::MODE_BF16>(make_params<float>(h, 0), V, q, fl, s);
    }
}

void free_handle(lbm_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->dT2) dev_free(h, h->dT2);
    if (h->cap) cudaStreamDestroy(h->cap);
    dev_free(h, h->base);
    if (h->stream && !h->release) cudaStreamSynchronize(h->stream);
    cudaGetLastError();
    delete h;
}

}  // namespace

extern "C" {

void lbm_params_default(lbm_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->nx = 150;
    p->ny = 150;
    p->thermal_q = 5;
    p->precision = LBM_F32;
    p->flow = 1;
    p->periodic_x = 0;
    p->periodic_y = 0;
    p->wall_kind[0] = LBM_WALL_DIRICHLET;
    p->wall_kind[1] = LBM_WALL_DIRICHLET;
    p->wall_kind[2] = LBM_WALL_ADIABATIC;
    p->wall_kind[3] = LBM_WALL_ADIABATIC;
    p->wall_T[0] = 1.0;
    p->wall_T[1] = 0.0;
    p->porosity = 0.8;
    p->Ra = 1e6;
    p->Pr = 50.0;
    p->Da = 1e-4;
    p->Ste = 1.0;
    p->cond_ratio = 1e3;
    p->Nu_i = 5.9;
    p->J = 1.0;
    p->F_phi = 0.068;
    p->sigma_hat = 1.0;
    p->dp_over_L = 0.0135;
    p->k_f = 5e-4;
    p->cfref_over_cpl = 0.2;
    p->cmref_over_cpm = 1.0;
    p->T_hot = 1.0;
    p->T_cold = 0.0;
    p->T_init = 0.0;
    p->T_ref0 = 0.0;
    p->T_solidus = 0.299;
    p->T_liquidus = 0.301;
    p->L_char = 150.0;
    p->varpi = 2.0 / 3.0;
    p->ks_over_kl = 1.0;
    p->cps_over_cpl = 1.0;
}

int lbm_derive(const lbm_params* p, lbm_derived* d) { return derive_impl(p, d); }

int64_t lbm_state_bytes(const lbm_params* p) {
    if (derive_impl(p, nullptr) != LBM_OK) return -1;
    return (int64_t)layout_of(*p).total;
}

int64_t lbm_history_bytes(const lbm_params* p) {
    if (derive_impl(p, nullptr) != LBM_OK) return -1;
    return (int64_t)layout_of(*p).dT_bytes;
}

int lbm_create_ex(const lbm_params* p, void* cuda_stream, lbm_alloc_fn alloc, lbm_free_fn release, void* ctx,
                  lbm_handle** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if ((alloc == nullptr) != (release == nullptr)) return LBM_ERR_ARG;
    lbm_derived d;
    int rc = derive_impl(p, &d);
    if (rc != LBM_OK) return rc;
    lbm_handle* h = new (std::nothrow) lbm_handle();
    if (!h) return LBM_ERR_OOM;
    h->p = *p;
    h->d = d;
    h->L = layout_of(*p);
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->alloc = alloc;
    h->release = release;
    h->ctx = ctx;
    h->base = static_cast<char*>(dev_alloc(h, h->L.total));
    if (!h->base) {
        delete h;
        return LBM_ERR_OOM;
    }
    h->buf[0] = h->base;
    h->buf[1] = h->base + h->L.off_buf1;
    h->dT = h->base + h->L.off_dT;
    h->status = reinterpret_cast<unsigned int*>(h->base + h->L.off_status);
    h->scratch = reinterpret_cast<double*>(h->base + h->L.off_scratch);
    h->diag_out = reinterpret_cast<double*>(h->base + h->L.off_out);
    // zero everything once: row padding is never written by the kernels, so
    // checkpoints of equal states are equal byte for byte
    cudaError_t e = cudaMemsetAsync(h->base, 0, h->L.total, h->stream);
    if (e == cudaSuccess) e = enqueue_init(h);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_handle(h);
        return LBM_ERR_CUDA;
    }
    *out = h;
    return LBM_OK;
}

int lbm_create(const lbm_params* p, void* cuda_stream, lbm_handle** out) {
    return lbm_create_ex(p, cuda_stream, nullptr, nullptr, nullptr, out);
}

int lbm_step(lbm_handle* h, int64_t nsteps) {
    if (!h || nsteps < 0) return LBM_ERR_ARG;
    if (h->sticky != LBM_OK) return h->sticky;
    int64_t n = nsteps;
    const bool two = two_steps(h);
    if (two && n >= 4) {
        const int rc = ensure_dT2(h);
        if (rc != LBM_OK) return rc;
    }
    while (n > 0 && h->cur != 0) {
        if (enqueue_one(h, h->cur, h->stream) != cudaSuccess) return cuda_fail(h);
        h->cur ^= 1;
        ++h->steps;
        --n;
    }
    if (n >= kGraphSteps) {
        int rc = build_graph(h);
        if (rc != LBM_OK) return rc;
        while (n >= kGraphSteps) {
            if (cudaGraphLaunch(h->graph, h->stream) != cudaSuccess) return cuda_fail(h);
            h->steps += kGraphSteps;
            n -= kGraphSteps;
        }
    }
    while (two && n >= 4) {   // two launches of two steps: copy and history back where they were
        if (enqueue_two(h, h->cur, 0, h->stream) != cudaSuccess || enqueue_two(h, h->cur ^ 1, 1, h->stream) != cudaSuccess)
            return cuda_fail(h);
        h->steps += 4;
        n -= 4;
    }
    while (n > 0) {
        if (enqueue_one(h, h->cur, h->stream) != cudaSuccess) return cuda_fail(h);
        h->cur ^= 1;
        ++h->steps;
        --n;
    }
    return h->sticky;
}

int lbm_step_form_for(const lbm_params* p, int32_t form, int32_t* used) {
    if (!p || !used || form < LBM_STEP_FORM_AUTO || form > LBM_STEP_FORM_TWO_STEPS) return LBM_ERR_ARG;
    const int rc = derive_impl(p, nullptr);
    if (rc != LBM_OK) return rc;
    const long long nodes = (long long)p->nx * p->ny;
    *used = lbmk::two_steps_for(p->precision, p->thermal_q, p->flow, nodes, form)
                ? LBM_STEP_FORM_TWO_STEPS
                : lbmk::form_for(p->precision, p->thermal_q, p->flow, p->solid_scheme, nodes, form);
    return LBM_OK;
}

int lbm_set_step_form(lbm_handle* h, int32_t form) {
    if (!h || form < LBM_STEP_FORM_AUTO || form > LBM_STEP_FORM_TWO_STEPS) return LBM_ERR_ARG;
    if (form != h->form && h->graph) {   // the captured steps used the old form
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h);
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    h->form = form;
    return LBM_OK;
}

int lbm_fields(lbm_handle* h, int32_t mask, void* const* dst, int32_t dst_on_device) {
    if (!h || !dst || (mask & ~((1 << LBM_NUM_FIELDS) - 1))) return LBM_ERR_ARG;
    if (h->sticky == LBM_ERR_CUDA) return LBM_ERR_STATE;
    for (int i = 0; i < LBM_NUM_FIELDS; ++i)
        if ((mask & (1 << i)) && !dst[i]) return LBM_ERR_ARG;
    if (!mask) return h->sticky;
    const size_t n = (size_t)h->p.nx * h->p.ny, bytes = n * h->L.relem;
    char* staging = nullptr;
    void* targets[LBM_NUM_FIELDS] = {nullptr};
    if (dst_on_device) {
        for (int i = 0; i < LBM_NUM_FIELDS; ++i) targets[i] = dst[i];
    } else {
        int cnt = 0;
        for (int i = 0; i < LBM_NUM_FIELDS; ++i) cnt += (mask >> i) & 1;
        staging = static_cast<char*>(dev_alloc(h, align_up(bytes) * cnt));
        if (!staging) return LBM_ERR_OOM;
        int k = 0;
        for (int i = 0; i < LBM_NUM_FIELDS; ++i)
            if (mask & (1 << i)) targets[i] = staging + align_up(bytes) * (k++);
    }
    cudaError_t e;
    const int q = h->p.thermal_q, fl = h->p.flow;
    if (h->p.precision == LBM_F64) {
        lbmk::FieldOut<double> o;
        for (int i = 0; i < 7; ++i) o.dst[i] = static_cast<double*>(targets[i]);
        o.mask = mask;
        o.ld = h->p.nx;
        e = lbmk::launch_fields<lbmk::MODE_F64>(make_params<double>(h, h->cur), o, q, fl, h->stream);
    } else {
        lbmk::FieldOut<float> o;
        for (int i = 0; i < 7; ++i) o.dst[i] = static_cast<float*>(targets[i]);
        o.mask = mask;
        o.ld = h->p.nx;
        const lbmk::StepParams<float> P = make_params<float>(h, h->cur);
        if (h->p.precision == LBM_F32) e = lbmk::launch_fields<lbmk::MODE_F32>(P, o, q, fl, h->stream);
        else if (h->p.precision == LBM_F16) e = lbmk::launch_fields<lbmk::MODE_F16>(P, o, q, fl, h->stream);
        else e = lbmk::launch_fields<lbmk::MODE_BF16>(P, o, q, fl, h->stream);
    }
    if (e == cudaSuccess && !dst_on_device)
        for (int i = 0; i < LBM_NUM_FIELDS && e == cudaSuccess; ++i)
            if (mask & (1 << i)) e = cudaMemcpyAsync(dst[i], targets[i], bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(h->stream);
        dev_free(h, staging);
        return cuda_fail(h);
    }
    int rc = sync_and_check(h);
    dev_free(h, staging);
    return rc;
}

int lbm_diag(lbm_handle* h, double* melt_frac, double* nu_hot, double* enthalpy, double* mass) {
    if (!h) return LBM_ERR_ARG;
    if (h->sticky == LBM_ERR_CUDA) return LBM_ERR_STATE;
    const lbm_params& p = h->p;
    lbmk::DiagConst C;
    C.phi = p.porosity;
    C.rho_l = 1.0;
    C.rho_m = h->d.rho_m;
    C.c_pm = 1.0;
    C.k_f = p.k_f;
    C.k_s = h->d.k_s;
    C.k_m = h->d.k_m;
    C.left_wall = (!p.periodic_x && p.nx >= 3) ? 1 : 0;
    cudaError_t e;
    const int q = p.thermal_q, fl = p.flow;
    if (p.precision == LBM_F64) {
        e = lbmk::launch_diag<lbmk::MODE_F64>(make_params<double>(h, h->cur), C, h->scratch, h->diag_out, q, fl,
                                              h->stream);
    } else {
        const lbmk::StepParams<float> P = make_params<float>(h, h->cur);
        if (p.precision == LBM_F32)
            e = lbmk::launch_diag<lbmk::MODE_F32>(P, C, h->scratch, h->diag_out, q, fl, h->stream);
        else if (p.precision == LBM_F16)
            e = lbmk::launch_diag<lbmk::MODE_F16>(P, C, h->scratch, h->diag_out, q, fl, h->stream);
        else
            e = lbmk::launch_diag<lbmk::MODE_BF16>(P, C, h->scratch, h->diag_out, q, fl, h->stream);
    }
    double s[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(s, h->diag_out, sizeof s, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h);
    int rc = sync_and_check(h);
    if (rc == LBM_ERR_CUDA) return rc;
    const double k_e = p.porosity * p.k_f + (1.0 - p.porosity) * h->d.k_m;
    if (melt_frac) *melt_frac = s[0] / ((double)p.nx * p.ny);
    if (nu_hot)
        *nu_hot = C.left_wall ? p.L_char / (k_e * (p.T_hot - p.T_cold)) * (s[3] / p.ny) : std::nan("");
    if (enthalpy) *enthalpy = s[1];
    if (mass) *mass = s[2];
    return rc;
}

// Copies the exchange history [ny][nx] in or out of its [ny][pitch] array.
static int copy_history(lbm_handle* h, void* host_or_dev, bool to_state, int on_device) {
    if (!host_or_dev) return LBM_OK;
    const size_t el = h->L.relem;
    const size_t dpitch = (size_t)h->p.nx * el, spitch = (size_t)h->L.pitch * el;
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : (to_state ? cudaMemcpyHostToDevice
                                                                           : cudaMemcpyDeviceToHost);
    cudaError_t e = to_state ? cudaMemcpy2DAsync(h->dT, spitch, host_or_dev, dpitch, dpitch, h->p.ny, kind, h->stream)
                             : cudaMemcpy2DAsync(host_or_dev, dpitch, h->dT, spitch, dpitch, h->p.ny, kind, h->stream);
    return e == cudaSuccess ? LBM_OK : cuda_fail(h);
}

// The state goes through dense arrays [q][ny][nx] of the run's arithmetic type
// on the device; the conversion kernel moves them to or from the chunked copy.
static int convert_state_io(lbm_handle* h, void* f, void* g, void* hm, void* lo, int to_state, int on_device) {
    const int Q = h->p.thermal_q;
    const size_t n = (size_t)h->p.nx * h->p.ny, el = h->L.relem;
    const size_t nf = h->p.flow ? 9 : 0;
    const bool has_lo = h->p.precision == LBM_F32;
    char* stage = static_cast<char*>(dev_alloc(h, align_up((nf + 2 * Q + (has_lo ? 1 : 0)) * n * el)));
    if (!stage) return LBM_ERR_OOM;
    void* Df = (h->p.flow && f) ? stage : nullptr;
    void* Dg = g ? stage + nf * n * el : nullptr;
    void* Dh = hm ? stage + (nf + Q) * n * el : nullptr;
    void* Dl = (has_lo && lo) ? stage + (nf + 2 * Q) * n * el : nullptr;
    const cudaMemcpyKind in = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind out = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaSuccess;
    if (to_state) {
        if (Df) e = cudaMemcpyAsync(Df, f, 9 * n * el, in, h->stream);
        if (e == cudaSuccess && Dg) e = cudaMemcpyAsync(Dg, g, Q * n * el, in, h->stream);
        if (e == cudaSuccess && Dh) e = cudaMemcpyAsync(Dh, hm, Q * n * el, in, h->stream);
        if (e == cudaSuccess && Dl) e = cudaMemcpyAsync(Dl, lo, n * el, in, h->stream);
    }
    if (e == cudaSuccess) {
        const int td = to_state ? 0 : 1;
        if (h->p.precision == LBM_F64) {
            lbmk::DenseState<double> D{static_cast<double*>(Df), static_cast<double*>(Dg), static_cast<double*>(Dh),
                                       nullptr};
            e = launch_convert_mode<lbmk::MODE_F64>(h, D, td);
        } else {
            lbmk::DenseState<float> D{static_cast<float*>(Df), static_cast<float*>(Dg), static_cast<float*>(Dh),
                                      static_cast<float*>(Dl)};
            if (h->p.precision == LBM_F32) e = launch_convert_mode<lbmk::MODE_F32>(h, D, td);
            else if (h->p.precision == LBM_F16) e = launch_convert_mode<lbmk::MODE_F16>(h, D, td);
            else e = launch_convert_mode<lbmk::MODE_BF16>(h, D, td);
        }
    }
    if (!to_state && e == cudaSuccess) {
        if (Df) e = cudaMemcpyAsync(f, Df, 9 * n * el, out, h->stream);
        if (e == cudaSuccess && Dg) e = cudaMemcpyAsync(g, Dg, Q * n * el, out, h->stream);
        if (e == cudaSuccess && Dh) e = cudaMemcpyAsync(hm, Dh, Q * n * el, out, h->stream);
        if (e == cudaSuccess && Dl) e = cudaMemcpyAsync(lo, Dl, n * el, out, h->stream);
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) e = cudaErrorUnknown;
    dev_free(h, stage);
    return e == cudaSuccess ? LBM_OK : cuda_fail(h);
}

int lbm_get_state(lbm_handle* h, void* f, void* g, void* hm, void* dT, void* g0_lo, int32_t on_device) {
    if (!h) return LBM_ERR_ARG;
    if (h->sticky == LBM_ERR_CUDA) return LBM_ERR_STATE;
    int rc = LBM_OK;
    if (f || g || hm || g0_lo) rc = convert_state_io(h, f, g, hm, g0_lo, 0, on_device);
    if (rc == LBM_OK) rc = copy_history(h, dT, false, on_device);
    if (rc != LBM_OK) return rc;
    return sync_and_check(h);
}

int lbm_set_state(lbm_handle* h, const void* f, const void* g, const void* hm, const void* dT, const void* g0_lo,
                  int32_t on_device) {
    if (!h) return LBM_ERR_ARG;
    if (h->sticky == LBM_ERR_CUDA) return LBM_ERR_STATE;
    int rc = LBM_OK;
    if (f || g || hm || g0_lo)
        rc = convert_state_io(h, const_cast<void*>(f), const_cast<void*>(g), const_cast<void*>(hm),
                              const_cast<void*>(g0_lo), 1, on_device);
    if (rc == LBM_OK) rc = copy_history(h, const_cast<void*>(dT), true, on_device);
    if (rc != LBM_OK) return rc;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h);
    return h->sticky;
}

namespace {
struct CkptHeader {
    char magic[8];
    int32_t version, precision, thermal_q, flow, nx, ny, pitch, nplanes;
    int64_t steps, copy_bytes, dT_bytes;
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header is 64 bytes");
const char kMagic[8] = {'L', 'B', 'M', 'C', 'K', 'P', 'T', '1'};

CkptHeader header_of(const lbm_handle* h) {
    CkptHeader c;
    std::memset(&c, 0, sizeof c);
    std::memcpy(c.magic, kMagic, 8);
    c.version = 2;   // 2: chunked state layout
    c.precision = h->p.precision;
    c.thermal_q = h->p.thermal_q;
    c.flow = h->p.flow;
    c.nx = h->p.nx;
    c.ny = h->p.ny;
    c.pitch = h->L.pitch;
    c.nplanes = h->L.nplanes;
    c.steps = h->steps;
    c.copy_bytes = (int64_t)h->L.copy_bytes;
    c.dT_bytes = (int64_t)h->L.dT_bytes;
    return c;
}
}  // namespace

int64_t lbm_checkpoint_bytes(const lbm_handle* h) {
    if (!h) return -1;
    return (int64_t)(sizeof(CkptHeader) + h->L.copy_bytes + h->L.dT_bytes);
}

int lbm_save(lbm_handle* h, void* dst, int32_t on_device) {
    if (!h || !dst) return LBM_ERR_ARG;
    if (h->sticky == LBM_ERR_CUDA) return LBM_ERR_STATE;
    const CkptHeader c = header_of(h);
    char* out = static_cast<char*>(dst);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = on_device ? cudaMemcpyAsync(out, &c, sizeof c, cudaMemcpyHostToDevice, h->stream)
                              : cudaSuccess;
    if (!on_device) std::memcpy(out, &c, sizeof c);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out + sizeof c, h->buf[h->cur], h->L.copy_bytes, k, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out + sizeof c + h->L.copy_bytes, h->dT, h->L.dT_bytes, k, h->stream);
    if (e != cudaSuccess) return cuda_fail(h);
    return sync_and_check(h);
}

int lbm_load(lbm_handle* h, const void* src, int32_t on_device) {
    if (!h || !src) return LBM_ERR_ARG;
    if (h->sticky == LBM_ERR_CUDA) return LBM_ERR_STATE;
    CkptHeader c;
    if (on_device) {
        if (cudaMemcpy(&c, src, sizeof c, cudaMemcpyDeviceToHost) != cudaSuccess) return cuda_fail(h);
    } else {
        std::memcpy(&c, src, sizeof c);
    }
    const CkptHeader want = header_of(h);
    if (std::memcmp(c.magic, kMagic, 8) != 0 || c.version != 2 || c.precision != want.precision ||
        c.thermal_q != want.thermal_q || c.flow != want.flow || c.nx != want.nx || c.ny != want.ny ||
        c.pitch != want.pitch || c.nplanes != want.nplanes || c.copy_bytes != want.copy_bytes ||
        c.dT_bytes != want.dT_bytes || c.steps < 0)
        return LBM_ERR_ARG;
    const char* in = static_cast<const char*>(src);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(h->buf[h->cur], in + sizeof c, h->L.copy_bytes, k, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->dT, in + sizeof c + h->L.copy_bytes, h->L.dT_bytes, k, h->stream);
    if (e != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h);
    h->steps = c.steps;
    return h->sticky;
}

int lbm_status(lbm_handle* h) {
    if (!h) return LBM_ERR_ARG;
    return sync_and_check(h);
}

int64_t lbm_steps_done(const lbm_handle* h) { return h ? h->steps : -1; }

int lbm_describe(const lbm_handle* h, lbm_params* p, lbm_derived* d) {
    if (!h) return LBM_ERR_ARG;
    if (p) *p = h->p;
    if (d) *d = h->d;
    return LBM_OK;
}

int lbm_destroy(lbm_handle* h) {
    if (!h) return LBM_OK;
    free_handle(h);
    return LBM_OK;
}

const char* lbm_strerror(int code) {
    switch (code) {
        case LBM_OK: return "ok";
        case LBM_ERR_ARG: return "invalid argument";
        case LBM_ERR_STABILITY: return "parameters outside the stable range of the scheme";
        case LBM_ERR_OOM: return "device allocation failed";
        case LBM_ERR_CUDA: return "CUDA runtime error";
        case LBM_ERR_UNSTABLE: return "non-finite or runaway state detected on the device";
        case LBM_ERR_TIMEOUT: return "bounded device wait expired";
        case LBM_ERR_STATE: return "handle in a failed state or call out of order";
        case LBM_ERR_TOO_LARGE: return "grid larger than the static scratch of the allocation-free diagnostics";
        default: return "unknown status code";
    }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: many runs advanced by one launch per time step
// ---------------------------------------------------------------------------

struct lbm_batch {
    std::vector<lbm_handle*> runs;
    int precision = 0, qt = 0, flow = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    lbm_alloc_fn alloc = nullptr;
    lbm_free_fn release = nullptr;
    void* ctx = nullptr;
    char* dev = nullptr;          // params[n][2] then tiles
    size_t params_stride = 0;     // bytes of one StepParams
    void* params = nullptr;
    std::vector<int> flip;        // run's current copy relative to the batch parity
    std::vector<int> form;        // each run's step form when the parameters were uploaded
    std::vector<int> shape;       // map 3: block shape of each run (index into kShapes)
    std::vector<std::vector<int>> groups;   // map 4: the runs of each grouped launch
    std::vector<int> solo;                  // map 4: runs that keep their own step kernel
    lbmk::Tile* tiles = nullptr;
    size_t tile_capacity = 0;     // tiles that fit in the allocation
    int ntiles = 0, width_cap = 128, chunk = 1, grid = 0, parity = 0, mapping = 0;
    double tuned_us = 0.0;
    cudaGraphExec_t graph = nullptr;
};

namespace {

// Block shapes of the single-run kernel under map 3 (threads in x, in y).
constexpr int kNumShapes = 9;
constexpr int kShapes[kNumShapes][2] = {{128, 2}, {64, 4}, {32, 8}, {256, 1}, {128, 1},
                                        {64, 2},  {32, 4}, {64, 1},  {32, 2}};
constexpr int kNumClasses = 4;

// Size class of a run for the shape tuner: by grid width, <= 64, <= 128, <= 256, wider.
int width_class(const lbm_handle* h) {
    const int nx = h->p.nx;
    return nx <= 64 ? 0 : (nx <= 128 ? 1 : (nx <= 256 ? 2 : 3));
}

int pow2_at_least(int v) {
    int p = 32;
    while (p < v && p < 256) p <<= 1;
    return p;
}

std::vector<lbmk::Tile> make_tiles(const std::vector<lbm_handle*>& runs, const std::vector<int>& flip,
                                   int width_cap) {
    std::vector<lbmk::Tile> t;
    for (int r = 0; r < (int)runs.size(); ++r) {
        const int nx = runs[r]->p.nx, ny = runs[r]->p.ny;
        const int w = std::min(width_cap, pow2_at_least(nx));
        int lg = 0;
        while ((1 << lg) < w) ++lg;
        const int h = 256 / w;
        const int code = lg | ((flip.empty() ? 0 : flip[r]) << 8);
        for (int y0 = 0; y0 < ny; y0 += h)
            for (int x0 = 0; x0 < nx; x0 += w) t.push_back({r, x0, y0, code});
    }
    return t;
}

void* batch_alloc(lbm_batch* b, size_t bytes, cudaStream_t s) {
    if (b->alloc) return b->alloc(bytes, b->ctx);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void batch_free(lbm_batch* b, void* p) {
    if (!p) return;
    if (b->release) b->release(p, b->ctx);
    else cudaFreeAsync(p, b->stream);
}

template <typename R>
void fill_params(lbm_batch* b, std::vector<char>& host) {
    for (size_t r = 0; r < b->runs.size(); ++r)
        for (int dir = 0; dir < 2; ++dir) {
            const lbmk::StepParams<R> P = make_params<R>(b->runs[r], dir);
            std::memcpy(host.data() + (2 * r + dir) * sizeof P, &P, sizeof P);
        }
}

// Writes the runs' parameter blocks ([run][direction]) and the tiles into b->dev.
int upload_batch(lbm_batch* b, const std::vector<lbmk::Tile>& tiles) {
    const size_t n = b->runs.size();
    if (tiles.size() > b->tile_capacity) return LBM_ERR_ARG;
    std::vector<char> host(2 * n * b->params_stride + tiles.size() * sizeof(lbmk::Tile));
    if (b->precision == LBM_F64) fill_params<double>(b, host);
    else fill_params<float>(b, host);
    std::memcpy(host.data() + 2 * n * b->params_stride, tiles.data(), tiles.size() * sizeof(lbmk::Tile));
    if (cudaMemcpyAsync(b->dev, host.data(), host.size(), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    b->params = b->dev;
    b->tiles = reinterpret_cast<lbmk::Tile*>(b->dev + 2 * n * b->params_stride);
    b->ntiles = (int)tiles.size();
    return LBM_OK;
}

// 1 when a run of the batch uses the Eq. 9 per-node rates (the tile kernel then
// compiles them in; runs without them still take their constant rates).
int batch_phase(const lbm_batch* b) {
    for (const lbm_handle* h : b->runs)
        if (phase_k_of(h)) return 1;
    return 0;
}

cudaError_t batch_launch(lbm_batch* b, int parity, cudaStream_t s) {
    const int q = b->qt, fl = b->flow, ph = batch_phase(b);
    const auto* pf = static_cast<const lbmk::StepParams<float>*>(b->params);
    switch (b->precision) {
        case LBM_F64:
            return lbmk::launch_batch<lbmk::MODE_F64>(static_cast<const lbmk::StepParams<double>*>(b->params),
                                                      b->tiles, b->ntiles, b->chunk, b->grid, parity, q, fl, ph, s);
        case LBM_F32:
            return lbmk::launch_batch<lbmk::MODE_F32>(pf, b->tiles, b->ntiles, b->chunk, b->grid, parity, q, fl, ph,
                                                      s);
        case LBM_F16:
            return lbmk::launch_batch<lbmk::MODE_F16>(pf, b->tiles, b->ntiles, b->chunk, b->grid, parity, q, fl, ph,
                                                      s);
        default:
            return lbmk::launch_batch<lbmk::MODE_BF16>(pf, b->tiles, b->ntiles, b->chunk, b->grid, parity, q, fl, ph,
                                                       s);
    }
}

int batch_blocks_per_sm(const lbm_batch* b) {
    const int ph = batch_phase(b);
    switch (b->precision) {
        case LBM_F64: return lbmk::batch_blocks_per_sm<lbmk::MODE_F64>(b->qt, b->flow, ph);
        case LBM_F32: return lbmk::batch_blocks_per_sm<lbmk::MODE_F32>(b->qt, b->flow, ph);
        case LBM_F16: return lbmk::batch_blocks_per_sm<lbmk::MODE_F16>(b->qt, b->flow, ph);
        default: return lbmk::batch_blocks_per_sm<lbmk::MODE_BF16>(b->qt, b->flow, ph);
    }
}

// Cell-to-block maps: 0 one block per tile, 1 persistent blocks over
// contiguous chunks of tiles, 2 persistent blocks striding over the tiles,
// 3 one single-run kernel per run and step, the runs' chains concurrent in
// one graph.
// Map 4: the runs below kGroupMaxNodes nodes in order, at most kGroupRuns per
// grouped launch; the larger runs keep their own step kernel.
// Map 4: the runs below kGroupMaxNodes in groups of at most kGroupRuns, the
// others solo.  Map 5: every run in groups (its kernel takes any size).
void make_groups(lbm_batch* b) {
    b->groups.clear();
    b->solo.clear();
    const int cap = b->precision == LBM_F64 ? lbmk::kGroupRuns<double> : lbmk::kGroupRuns<float>;
    std::vector<int> small;
    for (int r = 0; r < (int)b->runs.size(); ++r) {
        const lbm_params& p = b->runs[r]->p;
        if (b->mapping == 5 || (long long)p.nx * p.ny < lbmk::kGroupMaxNodes) small.push_back(r);
        else b->solo.push_back(r);
    }
    for (size_t i = 0; i < small.size(); i += cap)
        b->groups.emplace_back(small.begin() + i, small.begin() + std::min(small.size(), i + cap));
}

void set_mapping(lbm_batch* b, int mapping, int resident_blocks) {
    b->mapping = mapping;
    if (mapping == 4 || mapping == 5) make_groups(b);
    if (mapping >= 3) {
        b->grid = 0;
        b->chunk = 0;
    } else if (mapping == 0) {
        b->grid = b->ntiles;
        b->chunk = 1;
    } else {
        b->grid = std::max(1, std::min(b->ntiles, resident_blocks));
        b->chunk = mapping == 1 ? (b->ntiles + b->grid - 1) / b->grid : 0;
    }
}

void batch_destroy_graph(lbm_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

void free_batch(lbm_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_destroy_graph(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    batch_free(b, b->dev);
    if (b->stream) cudaStreamSynchronize(b->stream);
    cudaGetLastError();
    delete b;
}

// Adds to graph g one chain of `steps` step-kernel nodes for each listed run
// (the kernel, grid and block lbm_step would launch for the run, with the
// run's block shape), programmatic edges within a chain; a run's step k reads
// the copy flip ^ (k mod 2), starting from batch parity 0.
cudaError_t add_run_chains(lbm_batch* b, cudaGraph_t g, const std::vector<int>& which, int steps) {
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < which.size() && e == cudaSuccess; ++i) {
        const int r = which[i];
        lbm_handle* h = b->runs[r];
        cudaGraphNode_t prev = nullptr;
        for (int k = 0; k < steps && e == cudaSuccess; ++k) {
            const int from = b->flip[r] ^ (k & 1);
            lbmk::StepParams<double> Pd;
            lbmk::StepParams<float> Pf;
            void* args[1];
            if (b->precision == LBM_F64) {
                Pd = make_params<double>(h, from);
                args[0] = &Pd;
            } else {
                Pf = make_params<float>(h, from);
                args[0] = &Pf;
            }
            const dim3 blk((unsigned)kShapes[b->shape[r]][0], (unsigned)kShapes[b->shape[r]][1], 1u);
            lbmk::StepLaunch L;
            switch (b->precision) {   // the kernel and grid lbm_step would launch for this run
                case LBM_F64: L = lbmk::step_launch<lbmk::MODE_F64>(Pd, b->qt, b->flow, h->form, blk); break;
                case LBM_F32: L = lbmk::step_launch<lbmk::MODE_F32>(Pf, b->qt, b->flow, h->form, blk); break;
                case LBM_F16: L = lbmk::step_launch<lbmk::MODE_F16>(Pf, b->qt, b->flow, h->form, blk); break;
                default: L = lbmk::step_launch<lbmk::MODE_BF16>(Pf, b->qt, b->flow, h->form, blk); break;
            }
            cudaKernelNodeParams kp = {};
            kp.func = const_cast<void*>(L.fn);
            kp.gridDim = L.grid;
            kp.blockDim = L.block;
            kp.sharedMemBytes = 0;
            kp.kernelParams = args;
            kp.extra = nullptr;
            cudaGraphNode_t node = nullptr;
            e = cudaGraphAddKernelNode(&node, g, nullptr, 0, &kp);
            if (e == cudaSuccess && prev) {
                // programmatic edge, as lbm_step's launches: the next step of this
                // run launches while the previous one drains and waits for it
                // in-kernel before touching the state
                cudaGraphEdgeData ed = {};
                ed.from_port = cudaGraphKernelNodePortProgrammatic;
                ed.to_port = cudaGraphKernelNodePortDefault;
                ed.type = cudaGraphDependencyTypeProgrammatic;
                e = cudaGraphAddDependencies(g, &prev, &node, &ed, 1);
            }
            prev = node;
        }
    }
    return e;
}

int instantiate(cudaGraph_t g, cudaError_t e, cudaGraphExec_t* out) {
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    *out = exec;
    return LBM_OK;
}

// Map 3: a graph of `steps` steps with one chain of kernel nodes per run.
int build_chain_graph(lbm_batch* b, int steps, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return LBM_ERR_CUDA;
    std::vector<int> all(b->runs.size());
    for (size_t r = 0; r < all.size(); ++r) all[r] = (int)r;
    return instantiate(g, add_run_chains(b, g, all, steps), out);
}

// Maps 4 and 5: the parameters of one grouped launch -- its runs' parameter
// blocks for a step from batch parity `parity`, their tiles, and the prefix
// sums of their block counts.  two: a launch of the two-step kernel, whose
// history goes from h->dT to h->dT2 (back = 0) or back (back = 1).  Returns the
// launch's block count.
template <typename R>
long long fill_group(const lbm_batch* b, const std::vector<int>& g, int parity, lbmk::GroupParams<R>& G,
                     bool two, bool back) {
    std::memset(&G, 0, sizeof G);
    G.nruns = (int)g.size();
    long long acc = 0;
    for (size_t i = 0; i < g.size(); ++i) {
        lbm_handle* h = b->runs[g[i]];
        G.first_block[i] = (int)acc;
        G.run[i] = make_params<R>(h, b->flip[g[i]] ^ parity);
        if (two) {
            if (back) std::swap(G.run[i].dT, G.run[i].dT_out);
            acc += lbmk::group2_blocks(h->p.nx, h->p.ny);
        } else {
            G.tile[i] = lbmk::group_tile(h->p.nx);
            acc += lbmk::group_blocks(h->p.nx, h->p.ny, G.tile[i]);
        }
    }
    G.first_block[g.size()] = (int)acc;
    return acc;
}

const void* group_fn(const lbm_batch* b) {
    const int ph = batch_phase(b);
    switch (b->precision) {
        case LBM_F64: return lbmk::group_kernel<lbmk::MODE_F64>(b->qt, b->flow, ph);
        case LBM_F32: return lbmk::group_kernel<lbmk::MODE_F32>(b->qt, b->flow, ph);
        case LBM_F16: return lbmk::group_kernel<lbmk::MODE_F16>(b->qt, b->flow, ph);
        default: return lbmk::group_kernel<lbmk::MODE_BF16>(b->qt, b->flow, ph);
    }
}

// Map 5 applies to runs with flow in FP32/FP16/BF16 storage (the two-step kernel's).
bool two_step_batch(const lbm_batch* b) { return b->precision != LBM_F64 && b->flow; }

// The second history array of every run (map 5).
int ensure_batch_dT2(lbm_batch* b) {
    for (lbm_handle* h : b->runs) {
        const int rc = ensure_dT2(h);
        if (rc != LBM_OK) return rc;
    }
    return LBM_OK;
}

const void* group2_fn(const lbm_batch* b) {
    const int ph = batch_phase(b);
    switch (b->precision) {
        case LBM_F32: return lbmk::group2_kernel<lbmk::MODE_F32>(b->qt, ph);
        case LBM_F16: return lbmk::group2_kernel<lbmk::MODE_F16>(b->qt, ph);
        case LBM_BF16: return lbmk::group2_kernel<lbmk::MODE_BF16>(b->qt, ph);
        default: return nullptr;
    }
}

size_t group2_smem(const lbm_batch* b) {
    switch (b->precision) {
        case LBM_F32: return lbmk::step2_smem<lbmk::MODE_F32>(b->qt, lbmk::kT2HMany);
        case LBM_F16: return lbmk::step2_smem<lbmk::MODE_F16>(b->qt, lbmk::kT2HMany);
        case LBM_BF16: return lbmk::step2_smem<lbmk::MODE_BF16>(b->qt, lbmk::kT2HMany);
        default: return 0;
    }
}

// The launch configuration and the parameters of one grouped launch.
struct GroupArgs {
    std::unique_ptr<lbmk::GroupParams<double>> d;
    std::unique_ptr<lbmk::GroupParams<float>> f;
    void* args[1];
    dim3 grid, block;
    size_t smem = 0;
    const void* fn = nullptr;
};

cudaError_t group_args(const lbm_batch* b, const std::vector<int>& g, int parity, GroupArgs& a, bool two = false,
                       bool back = false) {
    long long blocks;
    if (b->precision == LBM_F64) {
        if (!a.d) a.d = std::make_unique<lbmk::GroupParams<double>>();
        blocks = fill_group<double>(b, g, parity, *a.d, false, false);
        a.args[0] = a.d.get();
    } else {
        if (!a.f) a.f = std::make_unique<lbmk::GroupParams<float>>();
        blocks = fill_group<float>(b, g, parity, *a.f, two, back);
        a.args[0] = a.f.get();
    }
    a.grid = dim3((unsigned)blocks, 1u, 1u);
    if (!two) {
        a.block = dim3(128, 1, 1);
        a.smem = 0;
        a.fn = group_fn(b);
        return cudaSuccess;
    }
    a.block = dim3((unsigned)lbmk::kT2W, (unsigned)lbmk::kT2HMany, 1u);
    a.smem = group2_smem(b);
    a.fn = group2_fn(b);
    if (!a.fn) return cudaErrorInvalidConfiguration;
    return cudaFuncSetAttribute(a.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.smem);
}

// One batched step under map 4 (each group's launch and each large run's
// own step) or two steps under map 5 (two = true: each group's two-step
// launch), as programmatic dependents of the previous launch in the stream.
// Single steps under map 5 take each run's one-step kernel (one node per
// thread), which rounds exactly as the two-step kernel does.
cudaError_t group_step_all(lbm_batch* b, int parity, cudaStream_t s, bool two = false, bool back = false) {
    if (b->mapping == 5 && !two) {
        for (size_t r = 0; r < b->runs.size(); ++r) {
            const cudaError_t e = enqueue_one(b->runs[r], b->flip[r] ^ parity, s, lbmk::FORM_SINGLE);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    GroupArgs a;
    for (const std::vector<int>& g : b->groups) {
        cudaError_t e = group_args(b, g, parity, a, two, back);
        if (e != cudaSuccess) return e;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = a.grid;
        cfg.blockDim = a.block;
        cfg.dynamicSmemBytes = a.smem;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelExC(&cfg, a.fn, a.args);
        if (e != cudaSuccess) return e;
    }
    for (int r : b->solo) {
        const cudaError_t e = enqueue_one(b->runs[r], b->flip[r] ^ parity, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Map 4: a graph of `steps` steps with one chain of grouped launches per group
// and one chain of step kernels per large run (programmatic edges within a
// chain; the chains are independent).  Map 5: steps / 2 two-step launches per
// group (steps even: copies and histories end where they started).
int build_group_graph(lbm_batch* b, int steps, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return LBM_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    GroupArgs a;
    const bool two = b->mapping == 5;
    const int launches = two ? steps / 2 : steps;
    for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) {
        cudaGraphNode_t prev = nullptr;
        for (int k = 0; k < launches && e == cudaSuccess; ++k) {
            e = group_args(b, b->groups[gi], k & 1, a, two, (k & 1) != 0);
            if (e != cudaSuccess) break;
            cudaKernelNodeParams kp = {};
            kp.func = const_cast<void*>(a.fn);
            kp.gridDim = a.grid;
            kp.blockDim = a.block;
            kp.sharedMemBytes = (unsigned)a.smem;
            kp.kernelParams = a.args;
            kp.extra = nullptr;
            cudaGraphNode_t node = nullptr;
            e = cudaGraphAddKernelNode(&node, g, nullptr, 0, &kp);
            if (e == cudaSuccess && prev) {
                cudaGraphEdgeData ed = {};
                ed.from_port = cudaGraphKernelNodePortProgrammatic;
                ed.to_port = cudaGraphKernelNodePortDefault;
                ed.type = cudaGraphDependencyTypeProgrammatic;
                e = cudaGraphAddDependencies(g, &prev, &node, &ed, 1);
            }
            prev = node;
        }
    }
    if (e == cudaSuccess) e = add_run_chains(b, g, b->solo, steps);
    return instantiate(g, e, out);
}

int build_batch_graph(lbm_batch* b) {
    if (b->graph) return LBM_OK;
    if (b->mapping == 4 || b->mapping == 5) return build_group_graph(b, kGraphSteps, &b->graph);
    if (b->mapping == 3) return build_chain_graph(b, kGraphSteps, &b->graph);
    if (!b->cap && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LBM_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < kGraphSteps && e == cudaSuccess; ++i) e = batch_launch(b, i & 1, b->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    cudaError_t e3 = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) {
        b->graph = nullptr;
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

// A run advanced by its own calls since the last batched step (lbm_step on
// the same stream, or after a synchronisation) may now read the other copy,
// and lbm_set_step_form may have changed its kernel.  Re-derive each run's
// copy relative to the batch parity; where anything moved, wait for the work
// in flight, rewrite the parameter blocks and the work list, and drop the
// replayed graph (map 3 bakes every run's copy and kernel into it).
int resync_runs(lbm_batch* b) {
    bool moved = false;
    for (size_t r = 0; r < b->runs.size(); ++r) {
        const int want = b->runs[r]->cur ^ b->parity;
        if (b->flip[r] != want || b->form[r] != b->runs[r]->form) moved = true;
        b->flip[r] = want;
        b->form[r] = b->runs[r]->form;
    }
    if (!moved) return LBM_OK;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    batch_destroy_graph(b);
    return upload_batch(b, make_tiles(b->runs, b->flip, b->width_cap));
}

int batch_advance(lbm_batch* b, int64_t n) {
    auto single = [&]() -> int {
        cudaError_t e = cudaSuccess;
        if (b->mapping == 4 || b->mapping == 5) {
            e = group_step_all(b, b->parity, b->stream);
        } else if (b->mapping == 3) {
            for (size_t r = 0; r < b->runs.size() && e == cudaSuccess; ++r)
                e = enqueue_one(b->runs[r], b->flip[r] ^ b->parity, b->stream);
        } else {
            e = batch_launch(b, b->parity, b->stream);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            return LBM_ERR_CUDA;
        }
        b->parity ^= 1;
        return LBM_OK;
    };
    int64_t left = n;
    while (left > 0 && b->parity != 0) {
        if (single() != LBM_OK) return LBM_ERR_CUDA;
        --left;
    }
    if (left >= kGraphSteps) {
        if (build_batch_graph(b) != LBM_OK) return LBM_ERR_CUDA;
        while (left >= kGraphSteps) {
            if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) {
                cudaGetLastError();
                return LBM_ERR_CUDA;
            }
            left -= kGraphSteps;
        }
    }
    while (b->mapping == 5 && left >= 4) {   // two two-step launches: copies and histories back in place
        if (group_step_all(b, b->parity, b->stream, true, false) != cudaSuccess ||
            group_step_all(b, b->parity ^ 1, b->stream, true, true) != cudaSuccess) {
            cudaGetLastError();
            return LBM_ERR_CUDA;
        }
        left -= 4;
    }
    while (left > 0) {
        if (single() != LBM_OK) return LBM_ERR_CUDA;
        --left;
    }
    return LBM_OK;
}

// Times `steps` batched steps of the current configuration (microseconds per step).
double time_batch(lbm_batch* b, int steps) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return 1e30;
    }
    cudaGraphExec_t g = nullptr;
    if ((b->mapping == 3 && build_chain_graph(b, steps, &g) != LBM_OK) ||
        ((b->mapping == 4 || b->mapping == 5) && build_group_graph(b, steps, &g) != LBM_OK)) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return 1e30;
    }
    if (g) cudaGraphLaunch(g, b->stream);
    else
        for (int i = 0; i < 4; ++i) batch_launch(b, i & 1, b->stream);
    cudaEventRecord(e0, b->stream);
    if (g) cudaGraphLaunch(g, b->stream);
    else
        for (int i = 0; i < steps; ++i) batch_launch(b, i & 1, b->stream);
    cudaEventRecord(e1, b->stream);
    if (g) {
        cudaStreamSynchronize(b->stream);
        cudaGraphExecDestroy(g);
    }
    float ms = 0.0f;
    const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    return ok ? 1e3 * ms / steps : 1e30;
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_handle* const* runs, int32_t n_runs, int32_t autotune, void* cuda_stream, lbm_batch** out) {
    if (!out || !runs || n_runs < 1) return LBM_ERR_ARG;
    *out = nullptr;
    for (int r = 0; r < n_runs; ++r) {
        if (!runs[r]) return LBM_ERR_ARG;
        if (runs[r]->sticky != LBM_OK) return LBM_ERR_STATE;
        if (runs[r]->p.precision != runs[0]->p.precision || runs[r]->p.thermal_q != runs[0]->p.thermal_q ||
            runs[r]->p.flow != runs[0]->p.flow)
            return LBM_ERR_ARG;
        for (int q = 0; q < r; ++q)
            if (runs[q] == runs[r]) return LBM_ERR_ARG;
    }
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_OOM;
    b->runs.assign(runs, runs + n_runs);
    b->precision = runs[0]->p.precision;
    b->qt = runs[0]->p.thermal_q;
    b->flow = runs[0]->p.flow;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->alloc = runs[0]->alloc;
    b->release = runs[0]->release;
    b->ctx = runs[0]->ctx;
    b->parity = 0;
    for (int r = 0; r < n_runs; ++r) {
        b->flip.push_back(runs[r]->cur);
        b->form.push_back(runs[r]->form);
    }
    // the single-run kernel's own shape rule until tuned (64 x 2 small, 128 x 1 large)
    for (int r = 0; r < n_runs; ++r) {
        const dim3 sb = lbmk::step_block(runs[r]->p.nx, runs[r]->p.ny);
        b->shape.push_back(sb.x == 64 ? 5 : 4);
    }
    b->params_stride = b->precision == LBM_F64 ? sizeof(lbmk::StepParams<double>) : sizeof(lbmk::StepParams<float>);
    for (lbm_handle* h : b->runs)
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return LBM_ERR_CUDA;
        }
    // room for the longest tile list any width cap gives (ragged widths make wide
    // tiles the longest list, narrow grids make narrow tiles the longest)
    size_t max_tiles = 0;
    for (int cap : {32, 64, 128, 256}) max_tiles = std::max(max_tiles, make_tiles(b->runs, b->flip, cap).size());
    b->tile_capacity = max_tiles;
    const size_t bytes = 2 * (size_t)n_runs * b->params_stride + max_tiles * sizeof(lbmk::Tile);
    b->dev = static_cast<char*>(batch_alloc(b, bytes, b->stream));
    if (!b->dev) {
        delete b;
        return LBM_ERR_OOM;
    }
    int dev_id = 0, sms = 0;
    cudaGetDevice(&dev_id);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    const int resident = std::max(1, batch_blocks_per_sm(b)) * std::max(1, sms);

    int best_cap = 128, best_map = 0;
    if (autotune) {
        // tune on fresh clones of the runs so the runs themselves do not move
        std::vector<lbm_handle*> clones;
        bool ok = true;
        for (lbm_handle* h : b->runs) {
            lbm_handle* c = nullptr;
            if (lbm_create_ex(&h->p, b->stream, h->alloc, h->release, h->ctx, &c) != LBM_OK) {
                ok = false;
                break;
            }
            c->form = h->form;   // time the kernels the runs themselves will take
            clones.push_back(c);
        }
        if (ok) {
            std::vector<lbm_handle*> keep = b->runs;
            b->runs = clones;
            b->parity = 0;
            double best = 1e30;
            std::vector<int> keep_flip(clones.size(), 0);   // fresh clones all start on copy 0
            b->flip.swap(keep_flip);
            // map 3: the block shape of each width class, by coordinate descent
            if (upload_batch(b, make_tiles(b->runs, b->flip, 128)) == LBM_OK) {
                set_mapping(b, 3, resident);
                double t3 = time_batch(b, 16);
                for (int c = 0; c < kNumClasses; ++c) {
                    std::vector<int> members;
                    for (size_t r = 0; r < b->runs.size(); ++r)
                        if (width_class(b->runs[r]) == c) members.push_back((int)r);
                    if (members.empty()) continue;
                    std::vector<int> start;   // the class's shapes before this pass
                    for (int r : members) start.push_back(b->shape[r]);
                    int chosen = -1;
                    for (int sh = 0; sh < kNumShapes; ++sh) {
                        for (int r : members) b->shape[r] = sh;
                        const double us = time_batch(b, 16);
                        if (us < t3) {
                            t3 = us;
                            chosen = sh;
                        }
                    }
                    for (size_t i = 0; i < members.size(); ++i) b->shape[members[i]] = chosen >= 0 ? chosen : start[i];
                }
                if (t3 < best) {
                    best = t3;
                    best_cap = 128;
                    best_map = 3;
                }
                set_mapping(b, 4, resident);
                const double t4 = time_batch(b, 16);
                if (t4 < best) {
                    best = t4;
                    best_cap = 128;
                    best_map = 4;
                }
                if (two_step_batch(b) && ensure_batch_dT2(b) == LBM_OK) {
                    set_mapping(b, 5, resident);
                    const double t5 = time_batch(b, 16);
                    if (t5 < best) {
                        best = t5;
                        best_cap = 128;
                        best_map = 5;
                    }
                }
            }
            for (int cap : {64, 128, 256}) {
                if (upload_batch(b, make_tiles(b->runs, b->flip, cap)) != LBM_OK) continue;
                for (int map = 0; map < 3; ++map) {
                    set_mapping(b, map, resident);
                    const double us = time_batch(b, 16);
                    if (us < best) {
                        best = us;
                        best_cap = cap;
                        best_map = map;
                    }
                }
            }
            b->flip.swap(keep_flip);
            b->tuned_us = best;
            b->runs = keep;
        }
        for (lbm_handle* c : clones) lbm_destroy(c);
        b->parity = 0;
    }
    b->width_cap = best_cap;
    if (upload_batch(b, make_tiles(b->runs, b->flip, best_cap)) != LBM_OK) {
        free_batch(b);
        return LBM_ERR_CUDA;
    }
    if (best_map == 5 && ensure_batch_dT2(b) != LBM_OK) best_map = 4;   // no room for the second histories
    set_mapping(b, best_map, resident);
    *out = b;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int64_t nsteps) {
    if (!b || nsteps < 0) return LBM_ERR_ARG;
    for (lbm_handle* h : b->runs)
        if (h->sticky != LBM_OK) return LBM_ERR_STATE;
    int rc = resync_runs(b);
    if (rc == LBM_OK) rc = batch_advance(b, nsteps);
    for (size_t r = 0; r < b->runs.size(); ++r) {
        lbm_handle* h = b->runs[r];
        h->cur = b->flip[r] ^ b->parity;
        if (rc == LBM_OK) h->steps += nsteps;
        else h->sticky = LBM_ERR_CUDA;
    }
    return rc;
}

int lbm_batch_configure(lbm_batch* b, int32_t width_cap, int32_t mapping) {
    if (!b || (width_cap != 32 && width_cap != 64 && width_cap != 128 && width_cap != 256) || mapping < 0 ||
        mapping > 5 || (mapping == 5 && !two_step_batch(b)))
        return LBM_ERR_ARG;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    if (mapping == 5) {
        const int rc = ensure_batch_dT2(b);
        if (rc != LBM_OK) return rc;
    }
    batch_destroy_graph(b);
    const int rc = upload_batch(b, make_tiles(b->runs, b->flip, width_cap));
    if (rc != LBM_OK) return rc;
    b->width_cap = width_cap;
    int dev_id = 0, sms = 0;
    cudaGetDevice(&dev_id);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    set_mapping(b, mapping, std::max(1, batch_blocks_per_sm(b)) * std::max(1, sms));
    return LBM_OK;
}

int lbm_batch_info(const lbm_batch* b, int32_t* n_tiles, int32_t* width_cap, int32_t* mapping, int32_t* grid,
                   double* tuned_us_per_step) {
    if (!b) return LBM_ERR_ARG;
    if (n_tiles) *n_tiles = b->ntiles;
    if (width_cap) *width_cap = b->width_cap;
    if (mapping) *mapping = b->mapping;
    if (grid) *grid = b->grid;
    if (tuned_us_per_step) *tuned_us_per_step = b->tuned_us;
    return LBM_OK;
}

int lbm_batch_set_block(lbm_batch* b, int32_t run, int32_t block_x, int32_t block_y) {
    if (!b || run < 0 || run >= (int32_t)b->runs.size()) return LBM_ERR_ARG;
    int id = -1;
    for (int k = 0; k < kNumShapes; ++k)
        if (kShapes[k][0] == block_x && kShapes[k][1] == block_y) id = k;
    if (id < 0) return LBM_ERR_ARG;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    batch_destroy_graph(b);
    b->shape[run] = id;
    return LBM_OK;
}

int lbm_batch_get_block(const lbm_batch* b, int32_t run, int32_t* block_x, int32_t* block_y) {
    if (!b || run < 0 || run >= (int32_t)b->runs.size()) return LBM_ERR_ARG;
    if (block_x) *block_x = kShapes[b->shape[run]][0];
    if (block_y) *block_y = kShapes[b->shape[run]][1];
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch* b) {
    free_batch(b);
    return LBM_OK;
}

}  // extern "C"
