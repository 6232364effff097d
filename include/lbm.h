/*
 * lbm.h -- C ABI of the GB300 enthalpy-based MRT lattice Boltzmann solver for
 * solid-liquid phase change in metal foams under local thermal
 * non-equilibrium (Liu, He & Li, arXiv 1701.00702).
 *
 * One call advances a run by whole time steps of the paper's fused
 * three-lattice update (Sec. III): a D2Q9 MRT flow lattice under the
 * generalized non-Darcy model (Eqs. 1-4, 12-27) with the volumetric solid
 * scheme (Eq. 20), and two MRT thermal lattices (D2Q5 of App. B by default,
 * or the D2Q9 of Sec. III B) for the PCM enthalpy (Eqs. 28-40) and the metal
 * foam internal energy (Eqs. 41-49), coupled by interstitial heat exchange
 * with its time-derivative correction (Eqs. 36, 47, Remark III).  The liquid
 * fraction follows from the enthalpy without iteration (Eqs. 37-39).  Walls
 * use non-equilibrium extrapolation (Eq. 52).
 *
 * Conventions shared by every entry point
 *  - Lattice units: delta_x = delta_t = c = 1, rho_l = 1, c_pl = c_ps = c_pm = 1
 *    (Sec. IV).  Grid nodes are (x, y), 0 <= x < nx, 0 <= y < ny; gravity
 *    points along -y.
 *  - Array layout at the boundary: every field is row-major [ny][nx] (x fastest);
 *    distribution arrays are [q][ny][nx] with the velocity order of Eq. 11
 *    (D2Q9: rest, +x, +y, -x, -y, (+,+), (-,+), (-,-), (+,-); D2Q5: the first
 *    five).  Element type is double for LBM_F64 runs and float for the others.
 *  - Status: every int-returning call returns LBM_OK (0) or a negative
 *    LBM_ERR_* code.  lbm_strerror() names it.  No call aborts the process.
 *  - Streams: work is enqueued on the cudaStream_t given at creation; calls
 *    that hand results to the host synchronise that stream first.
 *  - Threads: one handle must not be used from two threads at once; separate
 *    handles are independent.
 */
#ifndef PAPER_1701_00702_LBM_H
#define PAPER_1701_00702_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define LBM_OK             0
#define LBM_ERR_ARG       (-1)  /* bad argument: grid, porosity, null pointer, mask ... */
#define LBM_ERR_STABILITY (-2)  /* a derived relaxation rate or exchange rate is outside its stable range */
#define LBM_ERR_OOM       (-3)  /* device allocation failed */
#define LBM_ERR_CUDA      (-4)  /* a CUDA runtime call failed */
#define LBM_ERR_UNSTABLE  (-5)  /* the kernel saw a non-finite state or |u| > 0.3 (sticky) */
#define LBM_ERR_TIMEOUT   (-6)  /* a bounded device wait expired */
#define LBM_ERR_STATE     (-7)  /* handle already failed, or call out of order */
#define LBM_ERR_TOO_LARGE (-8)  /* grid exceeds the static scratch of lbm_diag_fields_noalloc */

/* ---- storage precision (lbm_params.precision) ----
 * LBM_F64   all populations FP64, FP64 arithmetic.
 * LBM_F32   all populations FP32, FP32 arithmetic; the PCM rest population is
 *           kept as a float-float pair (one extra FP32 plane) so that the
 *           enthalpy is conserved exactly.
 * LBM_F16, LBM_BF16  flow deviations f_i - w_i and the moving thermal
 *           populations in FP16 / BF16, the two thermal rest populations and
 *           the exchange history in FP32, FP32 arithmetic.
 * Fields and state arrays at the boundary are double for LBM_F64 and float
 * for the other three. */
#define LBM_F64  0
#define LBM_F32  1
#define LBM_F16  2
#define LBM_BF16 3

/* ---- wall kinds (lbm_params.wall_kind[side]) ---- */
#define LBM_WALL_DIRICHLET 0    /* T_f = T_m = wall_T[side] on the wall nodes */
#define LBM_WALL_ADIABATIC 1    /* T copied from the inward neighbour (zero normal gradient) */

/* sides, index of wall_kind / wall_T */
#define LBM_SIDE_LEFT   0       /* x = 0      */
#define LBM_SIDE_RIGHT  1       /* x = nx - 1 */
#define LBM_SIDE_BOTTOM 2       /* y = 0      */
#define LBM_SIDE_TOP    3       /* y = ny - 1 */

/* ---- field selection for lbm_fields (bit i selects dst[i]) ---- */
#define LBM_FIELD_T_F  (1 << 0)  /* PCM temperature T_f, Eq. 38 */
#define LBM_FIELD_T_S  (1 << 1)  /* metal-foam temperature T_m, Eq. 48 */
#define LBM_FIELD_F_L  (1 << 2)  /* liquid fraction f_l, Eq. 39 */
#define LBM_FIELD_U_X  (1 << 3)  /* velocity, Eq. 23 (0 on wall nodes) */
#define LBM_FIELD_U_Y  (1 << 4)
#define LBM_FIELD_RHO  (1 << 5)  /* density, Eq. 21 (1 when the flow lattice is off) */
#define LBM_FIELD_H_F  (1 << 6)  /* PCM enthalpy, Eq. 37 */
#define LBM_NUM_FIELDS 7

/*
 * Run description.  The non-dimensional groups are those of Eq. 54; their
 * map to lattice units (ν_f = Pr k_f, gβ = Ra ν_f k_f /(ΔT L³), K = Da L²,
 * k_m = λ k_f, ρ_m = σ̂, L_a = ΔT/Ste, h_v = Nu_i k_f / d_p², d_p = (d_p/L) L,
 * α_f,ref = k_f / c_f,ref, α_m,ref = k_m /(ρ_m c_m,ref)) and the relaxation
 * rates of Sec. III C and App. B are computed by lbm_derive().
 */
typedef struct lbm_params {
    int32_t nx, ny;            /* grid nodes; >= 3 in a direction that has walls */
    int32_t thermal_q;         /* 5 (App. B) or 9 (Sec. III B) */
    int32_t precision;         /* LBM_F64, LBM_F32, LBM_F16 or LBM_BF16 */
    int32_t flow;              /* 1: flow lattice on; 0: u = 0 everywhere (Sec. IV A) */
    int32_t periodic_x;        /* 1: periodic in x; 0: wall nodes at x = 0 and x = nx-1 */
    int32_t periodic_y;        /* 1: periodic in y; 0: wall nodes at y = 0 and y = ny-1 */
    int32_t wall_kind[4];      /* LBM_WALL_* per side (ignored on periodic sides) */
    double  wall_T[4];         /* Dirichlet wall temperatures per side */
    double  porosity;          /* φ, in (0, 1) */
    double  Ra, Pr, Da;        /* Rayleigh, Prandtl, Darcy numbers (Eq. 54) */
    double  Ste;               /* Stefan number St = c_pl ΔT / L_a */
    double  cond_ratio;        /* λ = k_m / k_f */
    double  Nu_i;              /* interstitial number H_v = h_v d_p² / k_f */
    double  J;                 /* ν_e / ν_f (paper: 1) */
    double  F_phi;             /* Forchheimer coefficient (paper: 0.068); < 0: Eq. 4's 1.75/sqrt(150 φ^3) */
    double  sigma_hat;         /* (ρc_p)_m / (ρc_p)_f (paper: 1) */
    double  dp_over_L;         /* pore size d_p / L (paper: 0.0135) */
    double  k_f;               /* PCM conductivity in lattice units (= α_f) */
    double  cfref_over_cpl;    /* c_f,ref / c_pl */
    double  cmref_over_cpm;    /* c_m,ref / c_pm */
    double  T_hot, T_cold;     /* ΔT = T_hot - T_cold (enters Ra and Ste) */
    double  T_init;            /* uniform initial temperature of both phases */
    double  T_ref0;            /* Boussinesq reference T_0 (Eq. 7) */
    double  T_solidus, T_liquidus;  /* T_fs <= T_fl (Eqs. 38-39) */
    double  L_char;            /* characteristic length L in lattice units */
    double  varpi;             /* ϖ of App. B, in (0, 1); used when thermal_q = 5 */
    /* comparison variants of Sec. V (0 = the present method) */
    int32_t thermal_collision; /* 0: MRT (Sec. III B); 1: BGK, every thermal rate = ζ_α (η_α) (Sec. V A) */
    int32_t solid_scheme;      /* 0: volumetric blend (Eq. 20); 1: bounce-back where f_l <= 0.5, no blend (Sec. V B) */
    double  zeta_e;            /* 0: ζ_e = 2 - ζ_α (Eq. 53); > 0: this ζ_e (and ζ_ε for D2Q9) instead (Sec. V D) */
    /* Phase-dependent PCM properties (Eq. 9): k_f = f_l k_l + (1 - f_l) k_s with
     * k_l = k_f above, and c_ps in Eq. 38.  With ks_over_kl != 1 every node
     * takes its own ζ_α (Eq. A19 at its liquid fraction) and ζ_e = 2 - ζ_α
     * (Eq. 53, unless zeta_e is given).  1 and 1 give the constant-property
     * method of Sec. IV. */
    double  ks_over_kl;        /* k_s / k_l, > 0 */
    double  cps_over_cpl;      /* c_ps / c_pl, > 0 */
} lbm_params;

/* Lattice-unit constants derived from lbm_params (output of lbm_derive). */
typedef struct lbm_derived {
    double nu_f, nu_e, gbeta, K, k_m, rho_m, L_a, d_p, h_v;
    double alpha_f, alpha_fref, alpha_mref, c_fref, c_mref, csT2;
    double H_fs, H_fl;         /* enthalpies at solidus and liquidus, Eqs. 38-39 */
    double l0, l1;             /* Eq. 25 */
    double exchange_rate;      /* h_v [1/(φ ρ_l) + 1/((1-φ) ρ_m)], must be < 1 */
    double s[9];               /* flow relaxation rates, Eq. 16 / Sec. III C */
    double zeta[9];            /* PCM rates Θ (first thermal_q entries) */
    double eta[9];             /* metal rates Q (first thermal_q entries) */
    double H_wall[4];          /* enthalpy of each Dirichlet wall, inverse of Eq. 38 */
    double k_s, c_ps;          /* solid PCM conductivity and specific heat (Eq. 9) */
    double zeta_a_solid;       /* ζ_α of a fully solid node (Eq. A19 with k_s); = zeta_a of liquid when k_s = k_l */
    double F_phi;              /* the Forchheimer coefficient in use (Eq. 4 when lbm_params.F_phi < 0) */
} lbm_derived;

typedef struct lbm_handle lbm_handle;

/* Allocation hooks: alloc returns 256-byte aligned device memory or NULL. */
typedef void* (*lbm_alloc_fn)(size_t bytes, void* ctx);
typedef void  (*lbm_free_fn)(void* ptr, void* ctx);

/* Fills p with the Sec. IV B square-cavity set-up on 150 x 150 (Ra = 1e6,
 * φ = 0.8, λ = 1e3, D2Q5 thermal lattices, FP32 storage).  Never fails. */
void lbm_params_default(lbm_params* p);

/* Validates p and computes the lattice constants (host only, no GPU needed).
 * Returns LBM_ERR_ARG for malformed input and LBM_ERR_STABILITY when a
 * relaxation rate leaves (0, 2), c_ref breaks Remark I (c_f,ref < 9/5 c_pf for
 * D2Q9, ϖ c_f,ref < c_pf for D2Q5; same for the metal) or the explicit
 * exchange rate reaches 1.  d may be NULL. */
int lbm_derive(const lbm_params* p, lbm_derived* d);

/* Device bytes a run will hold (two copies of the distributions, the exchange
 * history and small scratch).  A run that advances two steps per launch
 * (lbm_step in the two-step form, or a batch under map 5) adds a second
 * exchange-history array of lbm_history_bytes(p) at its first such step.  -1
 * if p is invalid. */
int64_t lbm_state_bytes(const lbm_params* p);

/* Device bytes of one exchange-history array of a run with parameters p (4
 * bytes per node of row pitch; 8 in FP64).  -1 if p is invalid. */
int64_t lbm_history_bytes(const lbm_params* p);

/* Creates a run, allocates its device state (through alloc/release when
 * given, else the CUDA stream-ordered allocator) and enqueues the uniform
 * initial state f = f^eq(1, 0), g = g^eq(H(T_init), T_init, 0),
 * h = h^eq(T_init) on cuda_stream (a cudaStream_t; NULL = legacy default
 * stream).  On failure *out is NULL and nothing stays allocated. */
int lbm_create(const lbm_params* p, void* cuda_stream, lbm_handle** out);
int lbm_create_ex(const lbm_params* p, void* cuda_stream, lbm_alloc_fn alloc,
                  lbm_free_fn release, void* ctx, lbm_handle** out);

/* Enqueues nsteps >= 0 time steps (Sec. III: stream, walls, enthalpy, blend,
 * velocity, three collisions).  Asynchronous: returns the sticky status known
 * on the host (LBM_ERR_UNSTABLE after any synchronising call saw the device
 * flag).  Large nsteps are replayed from a captured CUDA graph.  Each step is
 * launched as a programmatic dependent of the previous one in the stream.
 * The step kernel runs one node per thread in blocks of 64 x 2 threads on
 * grids of up to 40,000 nodes and 128 x 1 on larger ones, or node pairs, or
 * two steps per launch (see lbm_set_step_form). */
int lbm_step(lbm_handle* h, int64_t nsteps);

/* Step form of a run (the paper has no counterpart: an implementation
 * choice).  LBM_STEP_FORM_SINGLE: one node per thread.  LBM_STEP_FORM_PAIRS:
 * two neighbouring nodes per thread, each FP32 operation one packed
 * instruction for both; taken only by runs in the default configuration (flow,
 * D2Q5 thermal lattices, volumetric blend, FP32/FP16/BF16 storage), the others
 * keep one node per thread.  On grids of at least 1,572,864 nodes (state far
 * beyond L2) each node-pair block also asks L2 for the rows that blocks 48
 * rows further on will read (bulk L2 prefetch).  LBM_STEP_FORM_TWO_STEPS:
 * two time steps per launch for runs with flow in FP32/FP16/BF16 storage (the
 * others step one node per thread): each block of 34 x H threads advances its
 * tile and the one-node ring around it one step into shared memory, then the
 * tile's 32 x (H - 2) inner nodes a second step into the other state copy (H
 * from 4 to 16 per grid, at most two tiles per SM where the grid allows, else
 * H = 12);
 * lbm_step takes it for 4 steps or more (an odd remainder and steps that bring
 * the run back to state copy 0 are single steps).  LBM_STEP_FORM_AUTO (the
 * default), for runs with flow and the D2Q5 thermal lattices: two steps per
 * launch on grids of up to 102,400 nodes in FP32/FP16/BF16 and on FP32 grids
 * of at least 786,432 nodes (state beyond L2); node pairs for FP16/BF16 runs
 * of at least 1,572,864 (1536 x 1024) nodes; otherwise one node per thread.
 * Two steps per launch give the states of one step per launch bit for bit;
 * node pairs agree with them to within a few roundings of the FP32
 * arithmetic.  A run that steps two steps per launch keeps a second
 * exchange-history array (4 bytes per node of row pitch), allocated on the
 * run's allocator at the first lbm_step that uses the form (LBM_ERR_OOM if
 * that fails; nothing stepped).  Applies to later lbm_step calls and to
 * batches created afterwards (batches advance one step per launch: a run in
 * the two-step form steps there one node per thread); synchronises the run's
 * stream when it drops a captured graph.  LBM_ERR_ARG for another value. */
#define LBM_STEP_FORM_AUTO 0
#define LBM_STEP_FORM_SINGLE 1
#define LBM_STEP_FORM_PAIRS 2
#define LBM_STEP_FORM_TWO_STEPS 3
int lbm_set_step_form(lbm_handle* h, int32_t form);

/* The form (LBM_STEP_FORM_SINGLE, _PAIRS or _TWO_STEPS) a run with
 * parameters p steps in when set to `form`, written to *used.  Host only,
 * needs no GPU.  Returns lbm_derive's error for invalid p, LBM_ERR_ARG for
 * another form value or NULL pointers. */
int lbm_step_form_for(const lbm_params* p, int32_t form, int32_t* used);

/* Macroscopic fields at the current time level.  dst[i] receives field i of
 * LBM_FIELD_* when bit i of mask is set (nx*ny elements of the run's type,
 * [ny][nx]); dst_on_device selects device or host pointers.  Synchronises. */
int lbm_fields(lbm_handle* h, int32_t mask, void* const* dst, int32_t dst_on_device);

/* FP64 reductions at the current time level: melt fraction (mean f_l over all
 * nodes, Fig. 9), hot-wall Nusselt number (left-wall heat flux of both phases
 * by a second-order one-sided difference, times L/(k_e ΔT), k_e = φk_f+(1-φ)k_m),
 * total enthalpy Σ[φ ρ_l H_f + (1-φ) ρ_m c_pm T_m] and mass Σρ.  Any pointer
 * may be NULL.  Synchronises.  The reduction order is fixed, so equal states
 * give bit-equal results. */
int lbm_diag(lbm_handle* h, double* melt_frac, double* nu_hot, double* enthalpy, double* mass);

/* Copies the raw state out or in: f (9 planes; ignored when flow = 0), g and
 * hm (thermal_q planes each) hold the post-collision populations of the last
 * step, dT ([ny][nx]) the exchange history T_m - T_f of the last step.  The
 * flow populations are stored, and exchanged here, as deviations f_i - w_i
 * from the rest equilibrium f^eq(rho_0 = 1, u = 0) = w_i of Eq. 27
 * (w = 4/9, 1/9 x4, 1/36 x4); g and hm are the populations themselves.
 * With LBM_F32 storage the PCM rest population is the float-float sum
 * g[0] + g0_lo ([ny][nx]); g0_lo may be NULL (get: not copied; set: taken
 * as zero when g is given) and is ignored for the other modes.  LBM_F16 and
 * LBM_BF16 runs exchange the populations as float arrays: reading decodes the
 * stored form exactly, writing re-encodes with one 16-bit rounding per moving
 * population (use lbm_save / lbm_load for a bit-exact round trip).  Any other
 * pointer may be NULL to skip that array.  on_device selects device or host
 * pointers.  Synchronises. */
int lbm_get_state(lbm_handle* h, void* f, void* g, void* hm, void* dT, void* g0_lo, int32_t on_device);
int lbm_set_state(lbm_handle* h, const void* f, const void* g, const void* hm, const void* dT,
                  const void* g0_lo, int32_t on_device);

/* Raw checkpoints: the current state copy, the exchange history and the step
 * count, byte for byte, behind a 64-byte header that records the run's
 * layout.  lbm_load accepts only a checkpoint of a run with the same grid,
 * lattices, precision and flow flag (LBM_ERR_ARG otherwise) and restores it
 * bit for bit in every storage mode; the sticky status is left unchanged.
 * dst/src hold lbm_checkpoint_bytes(h) bytes on the device (on_device = 1)
 * or the host.  Both synchronise. */
int64_t lbm_checkpoint_bytes(const lbm_handle* h);
int lbm_save(lbm_handle* h, void* dst, int32_t on_device);
int lbm_load(lbm_handle* h, const void* src, int32_t on_device);

/* Synchronises the handle's stream and returns the sticky status. */
int lbm_status(lbm_handle* h);

/* Time steps taken so far. */
int64_t lbm_steps_done(const lbm_handle* h);

/* Copies the run's parameters and derived constants (either may be NULL). */
int lbm_describe(const lbm_handle* h, lbm_params* p, lbm_derived* d);

/* Synchronises, frees everything the handle owns.  NULL is a no-op. */
int lbm_destroy(lbm_handle* h);

/* Static string naming a status code. */
const char* lbm_strerror(int code);

/*
 * Batches: many runs (cavities of unequal size and parameters) advanced
 * together, replayed from CUDA graphs (the graph-launched form of Sec. III's
 * step for many independent problems; the paper itself runs one problem at
 * a time).
 *
 * lbm_batch_create takes n_runs distinct handles that share precision,
 * thermal_q and flow (their step counts may differ); it synchronises their
 * streams.  Maps 0-2 launch one kernel per time step over a list of tiles
 * (one run, w x 256/w nodes, w a power of two from 32 to 256): 0 one block
 * per tile, 1 persistent blocks over contiguous chunks of the list, 2
 * persistent blocks striding over the list.  Map 3 launches lbm_step's own
 * kernel once per run and step, each run a chain of kernel nodes in one
 * graph and the chains independent, so small runs overlap large ones; each
 * run's kernel takes one of the block shapes 128 x 2, 64 x 4, 32 x 8, 256 x 1
 * (256 threads), 128 x 1, 64 x 2, 32 x 4 (128) or 64 x 1, 32 x 2 (64).  Map
 * 4 steps the runs below 1,048,576 nodes in grouped launches, one kernel per
 * step for up to about 40 runs (23 in FP64) at a time, their parameter
 * blocks in the launch's own parameters, each run in tiles of w x 128/w
 * nodes (w = 32, 64 or 128, whichever leaves the fewest of the run's threads
 * idle); each group of runs is a chain of its own in the graph, and larger
 * runs keep their own step kernel in chains of their own, as under map 3.
 * Map 5 (runs with flow in FP32/FP16/BF16 storage) advances every run two
 * steps per launch in grouped launches of the two-step kernel (blocks of 34
 * x 12 threads, inner tiles of 32 x 10 nodes; see lbm_set_step_form), 32
 * launches per 64 steps, each run keeping a second exchange-history array
 * (allocated on its allocator when map 5 is chosen; LBM_ERR_OOM if that
 * fails); steps that align the batch to an even parity, and an odd
 * remainder, take each run's one-step kernel (one node per thread).
 * With autotune = 1 the call times, on freshly created copies of the runs (the
 * runs themselves do not move, but the copies hold as much device memory
 * again while tuning), map 3 with the block shape chosen per size class
 * (grid width <= 64, <= 128, <= 256, wider; one class at a time, keeping the
 * fastest shape), map 4, map 5 where it applies, and every combination of
 * tile-width cap (64, 128, 256) and map 0-2, and keeps the fastest; otherwise it takes width cap 128,
 * map 0, and for map 3 lbm_step's own block shapes (64 x 2 up to 40,000
 * nodes, 128 x 1 above).  Under map 3 a batched step equals lbm_step on each
 * run bit for bit.  Maps 0-2, 4 and 5 inline the same per-node code into
 * another kernel, where the compiler may fuse a few multiply-adds
 * differently: their states can differ from lbm_step's by a few roundings of
 * the arithmetic (FP32: 1-3 ulps in about 1e-4 of the flow populations per
 * step), which a 16-bit store sometimes carries into the last stored bit.  A
 * run's steps under maps 4 and 5 do not depend on the other runs of its
 * launch.
 *
 * lbm_batch_step enqueues nsteps steps of every run on the batch's stream
 * and advances each run's step count.  Use the runs' own calls (fields,
 * diagnostics, checkpoints, lbm_step, lbm_set_step_form) only on the same
 * stream or after synchronising it.  A run stepped by lbm_step between
 * batched steps holds its state in the other copy after an odd number of
 * steps; the next lbm_batch_step notices (as it notices a changed step form),
 * waits for the batch's stream, rewrites the parameter blocks and work list
 * and drops its replayed graph, then advances every run from its current
 * state.  A run whose sticky status is set stops the batch
 * (LBM_ERR_STATE).  lbm_batch_info reports the tile count, the chosen width
 * cap and map (0-5), the grid size (0 for maps 3-5) and the tuned
 * microseconds per step.
 * lbm_batch_destroy synchronises and frees the batch (not its runs).
 * The batch allocates its work list and parameter blocks through the first
 * run's allocation hooks (or the CUDA stream-ordered allocator).
 */
typedef struct lbm_batch lbm_batch;
int lbm_batch_create(lbm_handle* const* runs, int32_t n_runs, int32_t autotune, void* cuda_stream,
                     lbm_batch** out);
int lbm_batch_step(lbm_batch* b, int64_t nsteps);
/* Forces a tile-width cap (32, 64, 128 or 256) and a map (0-5; 5 only for
 * runs with flow in FP32/FP16/BF16 storage, LBM_ERR_ARG otherwise);
 * synchronises. */
int lbm_batch_configure(lbm_batch* b, int32_t width_cap, int32_t mapping);
int lbm_batch_info(const lbm_batch* b, int32_t* n_tiles, int32_t* width_cap, int32_t* mapping, int32_t* grid,
                   double* tuned_us_per_step);
/* Block shape of run `run` under map 3: one of the shapes listed above
 * (LBM_ERR_ARG otherwise).  The shape changes no result.  set synchronises
 * the batch's stream. */
int lbm_batch_set_block(lbm_batch* b, int32_t run, int32_t block_x, int32_t block_y);
int lbm_batch_get_block(const lbm_batch* b, int32_t run, int32_t* block_x, int32_t* block_y);
int lbm_batch_destroy(lbm_batch* b);

/*
 * Serving: continuous batching of melting runs.
 *
 * Requests (one lbm_params and a step count each) are queued by
 * lbm_server_submit.  Every lbm_server_tick
 *   1. admits queued requests in arrival order while fewer than max_active
 *      runs are active and the device bytes of the active runs
 *      (lbm_state_bytes, plus lbm_history_bytes under map 5) plus the next
 *      request's stay within hbm_budget_bytes;
 *   2. advances all active runs together by min(quantum, the smallest number
 *      of steps any active run still needs) through one lbm_batch (batched =
 *      1; the batch is rebuilt when membership changes, with the tile width
 *      cap and map of lbm_server_configure, default 128 and map 4, every
 *      active run in one grouped launch per step), then synchronises the
 *      stream;
 *   3. retires every run that has taken its steps: its FP64 diagnostics
 *      (lbm_diag) go into a result record and its device memory is freed.
 * A request that arrives while others run joins them at the next tick.
 * With batched = 0 the engine is the plain form: one request at a time, in
 * arrival order, each advanced by lbm_step.  A run's result is the same
 * alone and in the mix, bit for bit: under map 4 (the default) a run's steps
 * do not depend on the other runs of the launch, under map 3 they equal
 * lbm_step's.
 *
 * All requests of a server share precision, thermal_q and flow (LBM_ERR_ARG
 * otherwise); a request that the budget can never hold (its state, plus
 * its second history array under map 5) is refused at submission, or, if
 * the map changed after it was queued, at admission with status
 * LBM_ERR_ARG in its result.  lbm_server_configure takes maps 0-5 (5 only
 * for servers of runs with flow in FP32/FP16/BF16 storage).  Times in the results are seconds since lbm_server_create on
 * the host clock: submission, admission, completion.  lbm_server_results
 * moves up to max_results finished records into out.  lbm_server_stats
 * reports node updates performed, seconds the device was busy with ticks,
 * seconds since creation, and current and peak admitted bytes.  Device
 * memory comes through the allocation hooks (or the stream-ordered
 * allocator).  Not thread-safe.
 */
typedef struct lbm_request_result {
    int64_t id;
    int32_t status;            /* LBM_OK or the failure of this request */
    int32_t reserved;
    int64_t steps, nodes;      /* steps taken, grid nodes */
    double submit_s, admit_s, finish_s;
    double melt_frac, nu_hot, enthalpy, mass;   /* as lbm_diag, at the last step */
} lbm_request_result;

typedef struct lbm_server lbm_server;
int lbm_server_create(int64_t hbm_budget_bytes, int32_t max_active, int32_t batched, int32_t quantum,
                      int32_t precision, int32_t thermal_q, int32_t flow, void* cuda_stream, lbm_alloc_fn alloc,
                      lbm_free_fn release, void* ctx, lbm_server** out);
int lbm_server_configure(lbm_server* s, int32_t width_cap, int32_t mapping);
int lbm_server_submit(lbm_server* s, const lbm_params* p, int64_t nsteps, int64_t* id);
int lbm_server_tick(lbm_server* s, int32_t* n_active, int32_t* n_queued, int32_t* n_done);
int lbm_server_results(lbm_server* s, lbm_request_result* out, int32_t max_results, int32_t* n);
int lbm_server_stats(const lbm_server* s, int64_t* node_steps, double* busy_s, double* elapsed_s,
                     int64_t* used_bytes, int64_t* peak_used_bytes);
int lbm_server_destroy(lbm_server* s);

/*
 * Allocation-free diagnostics (the paper has no counterpart; this entry
 * point exists for callers that cannot allocate device memory).
 *
 * Who needs it: code whose device memory all belongs to another allocator (a
 * framework's memory pool, or a serving loop that has already handed out its
 * HBM budget) and latency-critical paths where cudaMalloc/cudaFree would
 * synchronise the device.  The call computes the four FP64 quantities of
 * lbm_diag -- out[0] melt fraction, out[1] hot-wall Nusselt number, out[2]
 * total enthalpy, out[3] mass -- from field arrays the caller already holds
 * (for instance written by lbm_fields with dst_on_device = 1), without a handle.
 * Precision: the sums are FP64, but they see only the fields as stored.  For
 * LBM_F64 the four values agree with lbm_diag to FP64 rounding.  For the
 * other modes the fields are FP32: out[0] and out[1] agree with lbm_diag to
 * FP64 rounding of the same FP32 values, while out[2] and out[3] carry about
 * 1e-7 relative error -- the H_f field is the high part of the PCM enthalpy
 * (lbm_diag adds the float-float low part of LBM_F32 and of Dirichlet wall
 * nodes) and rho is rounded to FP32 (lbm_diag sums 1 + (rho - 1)).  Use
 * lbm_diag for conservation-drift checks.
 *
 * Arguments: p describes the run (as for lbm_create); T_f, T_s, f_l, rho and
 * H_f are device arrays [ny][nx] of the run's element type (LBM_FIELD_* of
 * the same names); out is a device array of 4 doubles; cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  The work is enqueued on that
 * stream and the call returns without synchronising; the caller keeps
 * ownership of every buffer.
 *
 * Memory: no cudaMalloc, cudaFree or other allocating call is made.  The
 * per-block FP64 partial sums live in one file-scope device array of
 * 256 KiB (8192 blocks x 4 doubles) that every GPU loading this library
 * holds until the process exits; grids above LBM_DIAG_NOALLOC_MAX_NODES nodes
 * return LBM_ERR_TOO_LARGE.  Each call writes every partial it later reads,
 * so nothing has to start at zero.  All calls share that one array: calls
 * whose kernels overlap on the GPU (different streams, or different host
 * threads on the same device) race and give wrong sums; serialise them.
 *
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it together
 * with the ID of the device's current context; a call in a new context (after
 * cudaDeviceReset) looks it up again.  Make the first call on a device, and
 * the first call after a reset, before any stream capture.
 *
 * Errors: LBM_ERR_ARG for a null pointer or invalid p (LBM_ERR_STABILITY as
 * in lbm_derive), LBM_ERR_TOO_LARGE as above, LBM_ERR_CUDA if the symbol
 * lookup or a launch fails.
 */
#define LBM_DIAG_NOALLOC_MAX_NODES 67108864   /* 8192 x 8192 */
int lbm_diag_fields_noalloc(const lbm_params* p, const void* T_f, const void* T_s, const void* f_l,
                            const void* rho, const void* H_f, double* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* PAPER_1701_00702_LBM_H */
