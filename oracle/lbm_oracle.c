/*
 * Plain FP64 CPU oracle of the enthalpy-based MRT lattice Boltzmann step for
 * solid-liquid phase change in metal foams under local thermal
 * non-equilibrium (Liu, He & Li, arXiv 1701.00702).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path and is deliberately slow and literal:
 *   - lattice vectors come from Eq. 11 evaluated with cos/sin;
 *   - moments are dense products m = M f with the matrix typed in from
 *     Eq. 13 (D2Q9) or Eq. B1 (D2Q5), and f = M^-1 m with M^-1 obtained by
 *     Gauss-Jordan elimination at run time;
 *   - every node runs the steps of one time step in the paper's order:
 *       streaming (Eqs. 15, 33, 44) -> wall treatment (Eq. 52) ->
 *       enthalpy -> T_f, f_l (Eqs. 37-39), T_m (Eq. 48) ->
 *       volumetric solid blend (Eqs. 20-21) -> velocity (Eqs. 7, 23-25) ->
 *       flow MRT collision (Eqs. 3, 14, 18, 19) ->
 *       PCM enthalpy MRT collision (Eqs. 32, 34-36 or B2) ->
 *       metal MRT collision (Eqs. 43, 45-47 or B4).
 *
 * Readings taken where the paper is silent (each is a parameter of this
 * file, identical in the CUDA path, but implemented independently):
 *   - Wall nodes (Eq. 52): every population of a wall node is rebuilt from
 *     the state of the interior node x_f = x_b + inward normal (diagonal at
 *     corners); the wall velocity is u_b = 0 and the wall node collides with
 *     u = 0.  Temperatures: a Dirichlet wall sets T_f = T_m = T_wall and
 *     H = H(T_wall); an adiabatic wall copies T_f, H_f, T_m from x_f.  At a
 *     corner the x-wall (left/right) decides the temperature.
 *   - The source time derivative (Remark III) is the backward difference
 *     [Sr(t) - Sr(t-1)], so S = 1.5 Sr(t) - 0.5 Sr(t-1); the history is the
 *     per-node temperature gap dT = T_m - T_f of the previous step.
 *   - zeta_0 = eta_0 = 1 (they multiply n_0 - n_0^eq = 0 anyway).
 *   - D2Q5 (App. B): varpi is an input, zeta_e = 2 - zeta_alpha,
 *     zeta_epsilon = 1.2, eta_e = 1.1, eta_epsilon = 1.2 (set by the caller).
 *   - Comparison variants of Sec. V: BGK thermal collision is the rate vector
 *     with every entry zeta_alpha (eta_alpha), set by the caller; the
 *     bounce-back solid scheme (solid_scheme = 1) drops the blend of Eq. 20,
 *     treats nodes with f_l <= 0.5 as solid -- their arriving flow populations
 *     are sent back the way they came, f*_i = f+_opp(i), and u = 0 there --
 *     and collides the others with f = f+.
 *   - Phase-dependent PCM properties (Eq. 9): with phase_k = 1 the PCM
 *     conductivity is k_f = f_l k_l + (1 - f_l) k_s at the node's current
 *     liquid fraction, and the PCM rates that depend on it are rebuilt per
 *     node: zeta_alpha from Eq. A19, zeta_e = 2 - zeta_alpha (Eq. 53); which
 *     entries of the rate vector are which is set by the caller
 *     (zeta_role).  The specific heats c_ps, c_pl enter through Eq. 38.
 *
 * Storage: every distribution array is [q][ny][nx] (row-major, x fastest);
 * the stored values are the post-collision populations f*, g*, h* of the
 * previous step (the pre-streaming state).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct orc_cfg {
    int nx, ny;
    int qt;            /* thermal lattice size: 5 (App. B) or 9 (Sec. III B) */
    int flow;          /* 1: flow lattice evolved; 0: u = 0 everywhere */
    int periodic_x, periodic_y;
    int wall_kind[4];  /* 0 left, 1 right, 2 bottom, 3 top: 0 Dirichlet, 1 adiabatic */
    double wall_T[4];
    double phi, nu_f, K, F_phi, gbeta, T0;
    double rho_l, rho_m, c_pl, c_ps, c_pm, c_fref, c_mref, L_a, h_v;
    double T_fs, T_fl, varpi;
    double s[9];       /* flow relaxation diag, Eq. 16 */
    double zeta[9];    /* PCM relaxation diag, Theta (Eq. 31 / App. B) */
    double eta[9];     /* metal relaxation diag, Q (Eq. 42 / App. B) */
    int solid_scheme;  /* 0: volumetric blend (Eq. 20); 1: bounce-back where f_l <= 0.5 (Sec. V B, ref. 62) */
    int phase_k;       /* 1: PCM conductivity from Eq. 9 at each node, rates rebuilt per node */
    int zeta_role[9];  /* per PCM rate: 0 the fixed zeta[k], 1 zeta_alpha, 2 zeta_e = 2 - zeta_alpha */
    double k_l, k_s;   /* liquid and solid PCM conductivities (Eq. 9) */
    double csT2;       /* c_sT^2 of the thermal lattice (Eq. A19) */
} orc_cfg;

/* ------------------------------------------------------------------ */
/* Lattice (Eq. 11), weights (Eq. 27), transformation matrices         */
/* ------------------------------------------------------------------ */

static void lattice_vectors(int ex[9], int ey[9]) {
    for (int i = 0; i < 9; ++i) {
        double a, r;
        if (i == 0) { ex[i] = 0; ey[i] = 0; continue; }
        if (i <= 4) { a = (i - 1) * ORC_PI / 2.0; r = 1.0; }
        else { a = (2 * i - 9) * ORC_PI / 4.0; r = sqrt(2.0); }
        ex[i] = (int)lround(r * cos(a));
        ey[i] = (int)lround(r * sin(a));
    }
}

static double weight9(int i) {
    if (i == 0) return 4.0 / 9.0;
    if (i <= 4) return 1.0 / 9.0;
    return 1.0 / 36.0;
}

/* Eq. 13 */
static const double M9[81] = {
     1,  1,  1,  1,  1,  1,  1,  1,  1,
    -4, -1, -1, -1, -1,  2,  2,  2,  2,
     4, -2, -2, -2, -2,  1,  1,  1,  1,
     0,  1,  0, -1,  0,  1, -1, -1,  1,
     0, -2,  0,  2,  0,  1, -1, -1,  1,
     0,  0,  1,  0, -1,  1,  1, -1, -1,
     0,  0, -2,  0,  2,  1,  1, -1, -1,
     0,  1, -1,  1, -1,  0,  0,  0,  0,
     0,  0,  0,  0,  0,  1, -1,  1, -1,
};

/* Eq. B1 */
static const double M5[25] = {
    1,  1,  1,  1,  1,
    0,  1,  0, -1,  0,
    0,  0,  1,  0, -1,
    0,  1,  1,  1,  1,
    0,  1, -1,  1, -1,
};

/* Gauss-Jordan inverse with partial pivoting; returns 0 on success. */
static int invert(int n, const double* A, double* Ainv) {
    double W[9 * 18];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c)
            W[r * 2 * n + c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(W[r * 2 * n + col]) > fabs(W[piv * 2 * n + col])) piv = r;
        if (fabs(W[piv * 2 * n + col]) < 1e-300) return -1;
        if (piv != col)
            for (int c = 0; c < 2 * n; ++c) {
                double t = W[col * 2 * n + c];
                W[col * 2 * n + c] = W[piv * 2 * n + c];
                W[piv * 2 * n + c] = t;
            }
        double d = W[col * 2 * n + col];
        for (int c = 0; c < 2 * n; ++c) W[col * 2 * n + c] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double m = W[r * 2 * n + col];
            if (m == 0.0) continue;
            for (int c = 0; c < 2 * n; ++c) W[r * 2 * n + c] -= m * W[col * 2 * n + c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ainv[r * n + c] = W[r * 2 * n + n + c];
    return 0;
}

typedef struct tables {
    int ex[9], ey[9];
    double w[9];
    double Minv9[81], Minv5[25];
} tables;

static int make_tables(tables* t) {
    lattice_vectors(t->ex, t->ey);
    for (int i = 0; i < 9; ++i) t->w[i] = weight9(i);
    if (invert(9, M9, t->Minv9)) return -1;
    if (invert(5, M5, t->Minv5)) return -1;
    return 0;
}

static void matvec(int n, const double* A, const double* x, double* y) {
    for (int r = 0; r < n; ++r) {
        double s = 0.0;
        for (int c = 0; c < n; ++c) s += A[r * n + c] * x[c];
        y[r] = s;
    }
}

/* ------------------------------------------------------------------ */
/* Equilibria and sources                                              */
/* ------------------------------------------------------------------ */

#define CS2 (1.0 / 3.0)   /* c_s^2 = c^2/3 with c = 1 (D2Q9, Eq. 26) */

/* Eq. 27 */
static void f_eq(const orc_cfg* c, const tables* t, double rho, double ux, double uy, double* out) {
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double eu = t->ex[i] * ux + t->ey[i] * uy;
        out[i] = t->w[i] * rho * (1.0 + eu / CS2 + eu * eu / (2.0 * c->phi * CS2 * CS2)
                                  - uu / (2.0 * c->phi * CS2));
    }
}

/* Eq. 18 with alpha_1 = 1, alpha_2 = -3 */
static void m_eq(const orc_cfg* c, double rho, double ux, double uy, double* m) {
    double uu = ux * ux + uy * uy, p = c->phi;
    const double a1 = 1.0, a2 = -3.0;
    m[0] = rho;
    m[1] = rho * (-2.0 + 3.0 * uu / p);
    m[2] = rho * (a1 + a2 * uu / p);
    m[3] = rho * ux;
    m[4] = -rho * ux;
    m[5] = rho * uy;
    m[6] = -rho * uy;
    m[7] = rho * (ux * ux - uy * uy) / p;
    m[8] = rho * ux * uy / p;
}

/* Eq. 19 */
static void force_moments(const orc_cfg* c, double rho, double ux, double uy,
                          double Fx, double Fy, double* S) {
    double p = c->phi, uF = ux * Fx + uy * Fy;
    S[0] = 0.0;
    S[1] = rho * 6.0 * uF / p;
    S[2] = -rho * 6.0 * uF / p;
    S[3] = rho * Fx;
    S[4] = -rho * Fx;
    S[5] = rho * Fy;
    S[6] = -rho * Fy;
    S[7] = rho * 2.0 * (ux * Fx - uy * Fy) / p;
    S[8] = rho * (ux * Fy + uy * Fx) / p;
}

/* Eq. 40 (D2Q9) or Eq. B3 (D2Q5) */
static void g_eq(const orc_cfg* c, const tables* t, double H, double T, double ux, double uy, double* out) {
    if (c->qt == 9) {
        out[0] = H - 5.0 / 9.0 * c->c_fref * T;
        for (int i = 1; i < 9; ++i) {
            double eu = t->ex[i] * ux + t->ey[i] * uy;
            out[i] = t->w[i] * c->c_pl * T * (c->c_fref / c->c_pl + eu / (c->phi * CS2));
        }
    } else {
        double cst2 = c->varpi / 2.0;
        out[0] = H - c->varpi * c->c_fref * T;
        for (int i = 1; i < 5; ++i) {
            double eu = t->ex[i] * ux + t->ey[i] * uy;
            out[i] = 0.25 * c->varpi * c->c_pl * T * (c->c_fref / c->c_pl + eu / (c->phi * cst2));
        }
    }
}

/* Eq. 34 (D2Q9) or Eq. B2 (D2Q5) */
static void ng_eq(const orc_cfg* c, double H, double T, double ux, double uy, double* n) {
    double jx = c->c_pl * T * ux / c->phi, jy = c->c_pl * T * uy / c->phi;
    if (c->qt == 9) {
        n[0] = H;
        n[1] = -4.0 * H + 2.0 * c->c_fref * T;
        n[2] = 4.0 * H - 3.0 * c->c_fref * T;
        n[3] = jx; n[4] = -jx; n[5] = jy; n[6] = -jy;
        n[7] = 0.0; n[8] = 0.0;
    } else {
        n[0] = H; n[1] = jx; n[2] = jy; n[3] = c->varpi * c->c_fref * T; n[4] = 0.0;
    }
}

/* Eq. 49 (D2Q9) or Eq. B5 (D2Q5) */
static void h_eq(const orc_cfg* c, const tables* t, double Tm, double* out) {
    if (c->qt == 9) {
        out[0] = c->c_pm * Tm - 5.0 / 9.0 * c->c_mref * Tm;
        for (int i = 1; i < 9; ++i) out[i] = t->w[i] * c->c_mref * Tm;
    } else {
        out[0] = c->c_pm * Tm - c->varpi * c->c_mref * Tm;
        for (int i = 1; i < 5; ++i) out[i] = 0.25 * c->varpi * c->c_mref * Tm;
    }
}

/* Eq. 45 (D2Q9) or Eq. B4 (D2Q5) */
static void nh_eq(const orc_cfg* c, double Tm, double* n) {
    if (c->qt == 9) {
        n[0] = c->c_pm * Tm;
        n[1] = -4.0 * c->c_pm * Tm + 2.0 * c->c_mref * Tm;
        n[2] = 4.0 * c->c_pm * Tm - 3.0 * c->c_mref * Tm;
        for (int k = 3; k < 9; ++k) n[k] = 0.0;
    } else {
        n[0] = c->c_pm * Tm; n[1] = 0.0; n[2] = 0.0; n[3] = c->varpi * c->c_mref * Tm; n[4] = 0.0;
    }
}

/* Direction of the moment-space source: Eqs. 35, 46 (D2Q9); App. B (D2Q5) */
static void source_dir(const orc_cfg* c, double* s) {
    if (c->qt == 9) {
        for (int k = 0; k < 9; ++k) s[k] = 0.0;
        s[0] = 1.0; s[1] = -2.0; s[2] = 1.0;
    } else {
        s[0] = 1.0; s[1] = 0.0; s[2] = 0.0; s[3] = c->varpi; s[4] = 0.0;
    }
}

/* Eq. 38 */
/* PCM relaxation rates at a node of liquid fraction fl.  With phase_k the
 * conductivity follows Eq. 9, the reference diffusivity alpha_f,ref =
 * k_f/(rho_l c_f,ref) of Eq. A19 fixes zeta_alpha = 1/(1/2 + alpha_f,ref/c_sT^2),
 * and zeta_e = 2 - zeta_alpha (Eq. 53) where the caller asks for it. */
static void pcm_rates(const orc_cfg* c, double fl, double zeta[9]) {
    for (int k = 0; k < 9; ++k) zeta[k] = c->zeta[k];
    if (!c->phase_k) return;
    double kf = fl * c->k_l + (1.0 - fl) * c->k_s;                   /* Eq. 9 */
    double alpha_ref = kf / (c->rho_l * c->c_fref);                  /* Eq. A19 */
    double za = 1.0 / (0.5 + alpha_ref / c->csT2);
    for (int k = 0; k < 9; ++k) {
        if (c->zeta_role[k] == 1) zeta[k] = za;
        else if (c->zeta_role[k] == 2) zeta[k] = 2.0 - za;
    }
}

static double T_of_H(const orc_cfg* c, double H) {
    double Hfs = c->c_ps * c->T_fs, Hfl = c->c_pl * c->T_fl + c->L_a;
    if (H <= Hfs) return H / c->c_ps;
    if (H < Hfl) return c->T_fs + (H - Hfs) / (Hfl - Hfs) * (c->T_fl - c->T_fs);
    return c->T_fl + (H - Hfl) / c->c_pl;
}

/* Eq. 39 */
static double fl_of_H(const orc_cfg* c, double H) {
    double Hfs = c->c_ps * c->T_fs, Hfl = c->c_pl * c->T_fl + c->L_a;
    if (H <= Hfs) return 0.0;
    if (H < Hfl) return (H - Hfs) / (Hfl - Hfs);
    return 1.0;
}

/* Inverse of Eq. 38 used for Dirichlet walls and for the initial state:
 * T <= T_fs is solid, T >= T_fl (and > T_fs) is liquid, otherwise mushy. */
static double H_of_T(const orc_cfg* c, double T) {
    double Hfs = c->c_ps * c->T_fs, Hfl = c->c_pl * c->T_fl + c->L_a;
    if (T <= c->T_fs) return c->c_ps * T;
    if (T >= c->T_fl) return Hfl + c->c_pl * (T - c->T_fl);
    return Hfs + (T - c->T_fs) / (c->T_fl - c->T_fs) * (Hfl - Hfs);
}

/* Eqs. 23-25: explicit root of the velocity equation (22).  G = (0, Gy). */
static void velocity(const orc_cfg* c, double rho, double jx, double jy, double Gy,
                     double* ux, double* uy) {
    double vx = jx / rho;                             /* G_x = 0 */
    double vy = jy / rho + 0.5 * c->phi * Gy;
    double l0 = 0.5 * (1.0 + c->phi * 0.5 * c->nu_f / c->K);
    double l1 = c->phi * 0.5 * c->F_phi / sqrt(c->K);
    double vm = sqrt(vx * vx + vy * vy);
    double den = l0 + sqrt(l0 * l0 + l1 * vm);
    *ux = vx / den;
    *uy = vy / den;
}

/* ------------------------------------------------------------------ */
/* Node state                                                          */
/* ------------------------------------------------------------------ */

typedef struct node {
    double fp[9];   /* f^+ after streaming (and Eq. 52 at walls) */
    double f[9];    /* after the volumetric blend, Eq. 20 */
    double g[9], h[9];
    double rho, ux, uy, Gy, H, Tf, fl, Tm;
} node;

static int wrap(int i, int n, int periodic) {
    if (!periodic) return i;
    if (i < 0) return i + n;
    if (i >= n) return i - n;
    return i;
}

static size_t idx(const orc_cfg* c, int q, int x, int y) {
    return ((size_t)q * c->ny + y) * c->nx + x;
}

/* Streaming by pull: the population arriving at x along e_i left x - e_i. */
static void pull(const orc_cfg* c, const tables* t, const double* F, const double* G,
                 const double* Hh, int x, int y, node* n) {
    if (c->flow)
        for (int i = 0; i < 9; ++i) {
            int xs = wrap(x - t->ex[i], c->nx, c->periodic_x);
            int ys = wrap(y - t->ey[i], c->ny, c->periodic_y);
            n->fp[i] = F[idx(c, i, xs, ys)];
        }
    for (int i = 0; i < c->qt; ++i) {
        int xs = wrap(x - t->ex[i], c->nx, c->periodic_x);
        int ys = wrap(y - t->ey[i], c->ny, c->periodic_y);
        n->g[i] = G[idx(c, i, xs, ys)];
        n->h[i] = Hh[idx(c, i, xs, ys)];
    }
}

/* Thermal state from the distributions: Eqs. 37-39 and 48. */
static void thermal_state(const orc_cfg* c, node* n) {
    double H = 0.0, E = 0.0;
    for (int i = 0; i < c->qt; ++i) { H += n->g[i]; E += n->h[i]; }
    n->H = H;
    n->Tf = T_of_H(c, H);
    n->fl = fl_of_H(c, H);
    n->Tm = E / c->c_pm;
}

/* Eqs. 20-21 (blend), 7 (buoyancy), 23-25 (velocity).  The wall flag fixes u = u_b = 0. */
static void flow_state(const orc_cfg* c, const tables* t, node* n, int wall) {
    if (!c->flow) {
        n->rho = 1.0; n->ux = 0.0; n->uy = 0.0; n->Gy = 0.0;
        return;
    }
    double rho = 0.0;
    for (int i = 0; i < 9; ++i) rho += n->fp[i];
    if (c->solid_scheme == 1) {
        for (int i = 0; i < 9; ++i) n->f[i] = n->fp[i];
    } else {
        double fe0[9];
        f_eq(c, t, rho, 0.0, 0.0, fe0);
        for (int i = 0; i < 9; ++i) n->f[i] = n->fl * n->fp[i] + (1.0 - n->fl) * fe0[i];
    }
    n->rho = rho;
    n->Gy = c->gbeta * (n->Tf - c->T0) * n->fl;   /* G = -g beta (T_f - T_0) f_l, g along -y */
    if (wall || (c->solid_scheme == 1 && n->fl <= 0.5)) { n->ux = 0.0; n->uy = 0.0; return; }
    double jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) { jx += t->ex[i] * n->f[i]; jy += t->ey[i] * n->f[i]; }
    velocity(c, rho, jx, jy, n->Gy, &n->ux, &n->uy);
}

static int is_wall(const orc_cfg* c, int x, int y) {
    int wx = !c->periodic_x && (x == 0 || x == c->nx - 1);
    int wy = !c->periodic_y && (y == 0 || y == c->ny - 1);
    return wx || wy;
}

/* Full state of node (x, y) at the current time level. */
static void node_state(const orc_cfg* c, const tables* t, const double* F, const double* G,
                       const double* Hh, int x, int y, node* n) {
    if (!is_wall(c, x, y)) {
        pull(c, t, F, G, Hh, x, y, n);
        thermal_state(c, n);
        flow_state(c, t, n, 0);
        return;
    }
    /* Eq. 52: non-equilibrium extrapolation from the inward neighbour x_f. */
    int wx = !c->periodic_x && (x == 0 || x == c->nx - 1);
    int dx = !c->periodic_x ? (x == 0 ? 1 : (x == c->nx - 1 ? -1 : 0)) : 0;
    int dy = !c->periodic_y ? (y == 0 ? 1 : (y == c->ny - 1 ? -1 : 0)) : 0;
    node nf;
    pull(c, t, F, G, Hh, x + dx, y + dy, &nf);
    thermal_state(c, &nf);
    flow_state(c, t, &nf, 0);

    int side = wx ? (x == 0 ? 0 : 1) : (y == 0 ? 2 : 3);
    double Tb, Hb, Tmb;
    if (c->wall_kind[side] == 0) {
        Tb = c->wall_T[side]; Tmb = c->wall_T[side]; Hb = H_of_T(c, Tb);
    } else {
        Tb = nf.Tf; Hb = nf.H; Tmb = nf.Tm;
    }
    double a[9], b[9];
    if (c->flow) {
        f_eq(c, t, nf.rho, 0.0, 0.0, a);          /* \hat f^eq(rho(x_f), u_b = 0) */
        f_eq(c, t, nf.rho, nf.ux, nf.uy, b);       /* f^eq(x_f) */
        for (int i = 0; i < 9; ++i) n->fp[i] = a[i] + (nf.fp[i] - b[i]);
    }
    g_eq(c, t, Hb, Tb, 0.0, 0.0, a);
    g_eq(c, t, nf.H, nf.Tf, nf.ux, nf.uy, b);
    for (int i = 0; i < c->qt; ++i) n->g[i] = a[i] + (nf.g[i] - b[i]);
    h_eq(c, t, Tmb, a);
    h_eq(c, t, nf.Tm, b);
    for (int i = 0; i < c->qt; ++i) n->h[i] = a[i] + (nf.h[i] - b[i]);
    thermal_state(c, n);
    flow_state(c, t, n, 1);
}

/* Collision of the three lattices at one node; writes post-collision values. */
static void collide(const orc_cfg* c, const tables* t, const node* n, double dT_prev,
                    double* fs, double* gs, double* hs, double* dT_now) {
    if (c->flow && c->solid_scheme == 1 && n->fl <= 0.5) {
        /* bounce-back: each arriving population leaves along the opposite link */
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j)
                if (t->ex[j] == -t->ex[i] && t->ey[j] == -t->ey[i]) fs[i] = n->fp[j];
    } else if (c->flow) {
        /* Eq. 3 */
        double um = sqrt(n->ux * n->ux + n->uy * n->uy);
        double Fx = -c->phi * c->nu_f / c->K * n->ux - c->phi * c->F_phi / sqrt(c->K) * um * n->ux;
        double Fy = -c->phi * c->nu_f / c->K * n->uy - c->phi * c->F_phi / sqrt(c->K) * um * n->uy
                    + c->phi * n->Gy;
        double m[9], me[9], S[9], ms[9];
        matvec(9, M9, n->f, m);
        m_eq(c, n->rho, n->ux, n->uy, me);
        force_moments(c, n->rho, n->ux, n->uy, Fx, Fy, S);
        for (int k = 0; k < 9; ++k)                                    /* Eq. 14 */
            ms[k] = m[k] - c->s[k] * (m[k] - me[k]) + (1.0 - 0.5 * c->s[k]) * S[k];
        matvec(9, t->Minv9, ms, fs);
    }
    int Q = c->qt;
    const double* M = Q == 9 ? M9 : M5;
    const double* Mi = Q == 9 ? t->Minv9 : t->Minv5;
    double dir[9];
    source_dir(c, dir);

    double dT = n->Tm - n->Tf;
    /* Eqs. 36, 47 with the backward difference of Remark III */
    double Srf = c->h_v * dT / (c->phi * c->rho_l);
    double Srf_prev = c->h_v * dT_prev / (c->phi * c->rho_l);
    double S_pcm = Srf + 0.5 * (Srf - Srf_prev);
    double Srm = c->h_v * (-dT) / ((1.0 - c->phi) * c->rho_m);
    double Srm_prev = c->h_v * (-dT_prev) / ((1.0 - c->phi) * c->rho_m);
    double S_met = Srm + 0.5 * (Srm - Srm_prev);

    double zeta[9];
    pcm_rates(c, n->fl, zeta);
    double nv[9], ne[9], ns[9];
    matvec(Q, M, n->g, nv);                                            /* Eq. 32 */
    ng_eq(c, n->H, n->Tf, n->ux, n->uy, ne);
    for (int k = 0; k < Q; ++k) ns[k] = nv[k] - zeta[k] * (nv[k] - ne[k]) + S_pcm * dir[k];
    matvec(Q, Mi, ns, gs);

    matvec(Q, M, n->h, nv);                                            /* Eq. 43 */
    nh_eq(c, n->Tm, ne);
    for (int k = 0; k < Q; ++k) ns[k] = nv[k] - c->eta[k] * (nv[k] - ne[k]) + S_met * dir[k];
    matvec(Q, Mi, ns, hs);
    *dT_now = dT;
}

/* ------------------------------------------------------------------ */
/* Public entry points (called through ctypes)                         */
/* ------------------------------------------------------------------ */

int orc_check(const orc_cfg* c) {
    if (c->nx < 1 || c->ny < 1) return -1;
    if (c->qt != 5 && c->qt != 9) return -1;
    if (!c->periodic_x && c->nx < 3) return -1;
    if (!c->periodic_y && c->ny < 3) return -1;
    return 0;
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Uniform initial state: f = f^eq(rho0 = 1, 0), g = g^eq(H(T_i), T_i, 0), h = h^eq(T_i), dT = 0. */
int orc_init(const orc_cfg* c, double T_init, double* F, double* G, double* Hh, double* dT) {
    tables t;
    if (orc_check(c) || make_tables(&t)) return -1;
    double fe[9], ge[9], he[9];
    f_eq(c, &t, 1.0, 0.0, 0.0, fe);
    g_eq(c, &t, H_of_T(c, T_init), T_init, 0.0, 0.0, ge);
    h_eq(c, &t, T_init, he);
    size_t plane = (size_t)c->nx * c->ny;
    for (size_t k = 0; k < plane; ++k) {
        if (c->flow) for (int i = 0; i < 9; ++i) F[i * plane + k] = fe[i];
        for (int i = 0; i < c->qt; ++i) { G[i * plane + k] = ge[i]; Hh[i * plane + k] = he[i]; }
        dT[k] = 0.0;
    }
    return 0;
}

/* One time step: (F, G, Hh) -> (Fo, Go, Ho); dT is the per-node history, updated in place. */
int orc_step(const orc_cfg* c, const double* F, const double* G, const double* Hh,
             double* dT, double* Fo, double* Go, double* Ho) {
    tables t;
    if (orc_check(c) || make_tables(&t)) return -1;
    int nx = c->nx, ny = c->ny;
    size_t plane = (size_t)nx * ny;
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            node n;
            double fs[9], gs[9], hs[9], dTn;
            size_t k = (size_t)y * nx + x;
            node_state(c, &t, F, G, Hh, x, y, &n);
            collide(c, &t, &n, dT[k], fs, gs, hs, &dTn);
            if (c->flow) for (int i = 0; i < 9; ++i) Fo[i * plane + k] = fs[i];
            for (int i = 0; i < c->qt; ++i) { Go[i * plane + k] = gs[i]; Ho[i * plane + k] = hs[i]; }
            dT[k] = dTn;   /* each node reads and writes only its own entry */
        }
    }
    return 0;
}

/* Macroscopic fields at the current time level (state after streaming, walls, blend). */
int orc_fields(const orc_cfg* c, const double* F, const double* G, const double* Hh,
               double* Tf, double* Tm, double* fl, double* ux, double* uy, double* rho, double* H) {
    tables t;
    if (orc_check(c) || make_tables(&t)) return -1;
    int nx = c->nx, ny = c->ny;
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            node n;
            size_t k = (size_t)y * nx + x;
            node_state(c, &t, F, G, Hh, x, y, &n);
            Tf[k] = n.Tf; Tm[k] = n.Tm; fl[k] = n.fl;
            ux[k] = n.ux; uy[k] = n.uy; rho[k] = n.rho; H[k] = n.H;
        }
    return 0;
}

/* ---- single-formula entry points used by the pin tests ---- */

int orc_lattice(int* ex, int* ey, double* w) {
    lattice_vectors(ex, ey);
    for (int i = 0; i < 9; ++i) w[i] = weight9(i);
    return 0;
}

int orc_matrices(int q, double* M, double* Minv) {
    tables t;
    if (make_tables(&t)) return -1;
    if (q == 9) { memcpy(M, M9, sizeof M9); memcpy(Minv, t.Minv9, sizeof t.Minv9); return 0; }
    if (q == 5) { memcpy(M, M5, sizeof M5); memcpy(Minv, t.Minv5, sizeof t.Minv5); return 0; }
    return -1;
}

void orc_f_eq(const orc_cfg* c, double rho, double ux, double uy, double* out) {
    tables t; make_tables(&t); f_eq(c, &t, rho, ux, uy, out);
}
void orc_m_eq(const orc_cfg* c, double rho, double ux, double uy, double* out) { m_eq(c, rho, ux, uy, out); }
void orc_force_moments(const orc_cfg* c, double rho, double ux, double uy, double Fx, double Fy, double* S) {
    force_moments(c, rho, ux, uy, Fx, Fy, S);
}
void orc_g_eq(const orc_cfg* c, double H, double T, double ux, double uy, double* out) {
    tables t; make_tables(&t); g_eq(c, &t, H, T, ux, uy, out);
}
void orc_ng_eq(const orc_cfg* c, double H, double T, double ux, double uy, double* out) { ng_eq(c, H, T, ux, uy, out); }
void orc_h_eq(const orc_cfg* c, double Tm, double* out) { tables t; make_tables(&t); h_eq(c, &t, Tm, out); }
void orc_nh_eq(const orc_cfg* c, double Tm, double* out) { nh_eq(c, Tm, out); }
double orc_T_of_H(const orc_cfg* c, double H) { return T_of_H(c, H); }
double orc_fl_of_H(const orc_cfg* c, double H) { return fl_of_H(c, H); }
double orc_H_of_T(const orc_cfg* c, double T) { return H_of_T(c, T); }
void orc_velocity(const orc_cfg* c, double rho, double jx, double jy, double Gy, double* u) {
    velocity(c, rho, jx, jy, Gy, &u[0], &u[1]);
}

/* One time step evaluated only at the listed nodes (for sampled checks of
 * large grids): outputs are [n][9] (flow), [n][qt] (PCM, metal) and [n]. */
int orc_step_nodes(const orc_cfg* c, const double* F, const double* G, const double* Hh,
                   const double* dT, const int* xs, const int* ys, int n,
                   double* fo, double* go, double* ho, double* dTo) {
    tables t;
    if (orc_check(c) || make_tables(&t)) return -1;
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < n; ++k) {
        int x = xs[k], y = ys[k];
        if (x < 0 || x >= c->nx || y < 0 || y >= c->ny) continue;
        node nd;
        double fs[9], gs[9], hs[9], dTn;
        node_state(c, &t, F, G, Hh, x, y, &nd);
        collide(c, &t, &nd, dT[(size_t)y * c->nx + x], fs, gs, hs, &dTn);
        if (c->flow) for (int i = 0; i < 9; ++i) fo[(size_t)k * 9 + i] = fs[i];
        for (int i = 0; i < c->qt; ++i) { go[(size_t)k * c->qt + i] = gs[i]; ho[(size_t)k * c->qt + i] = hs[i]; }
        dTo[k] = dTn;
    }
    return 0;
}
