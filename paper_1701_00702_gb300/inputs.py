"""Seeded synthetic inputs: run parameters and initial states.

This module holds no arithmetic of the lattice Boltzmann method.  It only
writes down parameter sets (the paper's Sec. IV set-ups at the sizes the
benchmarks use) and draws seeded random numbers.  Both the CUDA path's tests
and the oracle's tests take their inputs from here.

Parameter dictionaries use the field names of the C ABI's ``lbm_params``
struct (``include/lbm.h``).  The paper's workloads are analytic set-ups
rather than datasets, so no public data stands behind any of them.
"""
from __future__ import annotations

import numpy as np

PREC_F64 = 0
PREC_F32 = 1
PREC_F16 = 2
PREC_BF16 = 3

WALL_DIRICHLET = 0
WALL_ADIABATIC = 1

DEFAULT_SEED = 1701


def paper_cavity_defaults() -> dict:
    """Sec. IV B: melting with natural convection in a square cavity heated from
    the left (T_h = 1), cooled on the right (T_c = 0), adiabatic top and bottom;
    phi = 0.8, Da = 1e-4, Pr = 50, F_phi = 0.068, lambda = 1e3, St = 1, J = 1,
    k_f = 5e-4, c_f,ref = 0.2 c_pl, c_m,ref = c_pm, T_fs/T_fl = 0.299/0.301,
    H_v = 5.9, d_p/L = 0.0135, sigma_hat = 1; Ra = 1e6 on 150 x 150."""
    return dict(
        nx=150, ny=150, thermal_q=5, precision=PREC_F32, flow=1,
        periodic_x=0, periodic_y=0,
        wall_kind=[WALL_DIRICHLET, WALL_DIRICHLET, WALL_ADIABATIC, WALL_ADIABATIC],
        wall_T=[1.0, 0.0, 0.0, 0.0],
        porosity=0.8, Ra=1e6, Pr=50.0, Da=1e-4, Ste=1.0, cond_ratio=1e3, Nu_i=5.9,
        J=1.0, F_phi=0.068, sigma_hat=1.0, dp_over_L=0.0135, k_f=5e-4,
        cfref_over_cpl=0.2, cmref_over_cpm=1.0,
        T_hot=1.0, T_cold=0.0, T_init=0.0, T_ref0=0.0, T_solidus=0.299, T_liquidus=0.301,
        L_char=150.0, varpi=2.0 / 3.0,
        thermal_collision=0, solid_scheme=0, zeta_e=0.0, ks_over_kl=1.0, cps_over_cpl=1.0,
    )


def cavity(n: int = 256, ny: int | None = None, precision: int = PREC_F32, thermal_q: int = 5,
           **over) -> dict:
    """Square-cavity melting (Sec. IV B set-up) with porosity 0.9 and
    conductivity ratio 100, L = n; Ra = 1e6, Pr = 50, Da = 1e-4, Ste = 1."""
    p = paper_cavity_defaults()
    p.update(nx=int(n), ny=int(ny if ny is not None else n), precision=precision, thermal_q=thermal_q,
             porosity=0.9, cond_ratio=100.0, L_char=float(n))
    p.update(over)
    return p


def conduction_1d(nx: int = 200, ny: int = 4, precision: int = PREC_F64, thermal_q: int = 5,
                  **over) -> dict:
    """Conduction-only LTNE melting (flow off, u = 0): hot left wall T = 1, right
    wall held at the initial T = 0, periodic in y; porosity 0.95, Ste = 1,
    conductivity ratio 100, interstitial H_v = 1; the Sec. IV A constants
    k_f = 0.01, L = nx/2, c_f,ref = 0.5, c_m,ref = 1; isothermal melting at
    T_melt = 0 (T_fs = T_fl = 0), initially solid at T = 0."""
    p = paper_cavity_defaults()
    p.update(nx=int(nx), ny=int(ny), precision=precision, thermal_q=thermal_q, flow=0,
             periodic_x=0, periodic_y=1,
             wall_kind=[WALL_DIRICHLET, WALL_DIRICHLET, WALL_ADIABATIC, WALL_ADIABATIC],
             wall_T=[1.0, 0.0, 0.0, 0.0],
             porosity=0.95, Ste=1.0, cond_ratio=100.0, Nu_i=1.0, k_f=0.01,
             cfref_over_cpl=0.5, cmref_over_cpm=1.0, T_hot=1.0, T_cold=0.0, T_init=0.0,
             T_solidus=0.0, T_liquidus=0.0, L_char=float(nx) / 2.0)
    p.update(over)
    return p


def heated_cavity(n: int, Ra: float, k_f: float = 0.05, precision: int = PREC_F64, **over) -> dict:
    """The differentially heated square cavity of natural convection, reached
    as a limit of the Sec. IV B set-up: porosity 0.9999, Da = 1e9 and
    F_phi = 0 (no porous drag), H_v = 0 (the metal lattice decouples),
    conductivity ratio 1, Pr = 0.71, and a melting point below the cold wall
    so that the PCM is liquid throughout.  Walls are the nodes x = 0 and
    x = n - 1, so the cavity width is L = n - 1; the run starts at the mean
    temperature 0.5, which is also the buoyancy reference."""
    p = cavity(n, precision=precision, porosity=0.9999, Nu_i=0.0, Da=1e9, F_phi=0.0, Pr=0.71,
               cond_ratio=1.0, Ra=float(Ra), T_solidus=-1.0, T_liquidus=-1.0, T_init=0.5, T_ref0=0.5,
               k_f=float(k_f), cfref_over_cpl=0.5, L_char=float(n - 1))
    p.update(over)
    return p


def periodic_box(nx: int, ny: int, **over) -> dict:
    """Fully periodic box (no walls): the set-up of the conservation checks."""
    p = cavity(max(nx, ny))
    p.update(nx=int(nx), ny=int(ny), periodic_x=1, periodic_y=1)
    p.update(over)
    return p


def batch_draws(count: int = 64, seed: int = DEFAULT_SEED, n_lo: int = 64, n_hi: int = 512) -> list[dict]:
    """Many unequal cavities: side drawn uniformly from [n_lo, n_hi], porosity
    uniform in [0.85, 0.98], Da and Ra log-uniform in [1e-5, 1e-3] and
    [1e4, 1e6], Ste uniform in [0.5, 2]; everything else as in ``cavity``."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        out.append(cavity(n,
                          porosity=float(rng.uniform(0.85, 0.98)),
                          Da=float(10 ** rng.uniform(-5, -3)),
                          Ra=float(10 ** rng.uniform(4, 6)),
                          Ste=float(rng.uniform(0.5, 2.0))))
    return out


def serving_arrivals(count: int, rate_per_s: float, seed: int = DEFAULT_SEED,
                     grids=((128, 128), (256, 256), (512, 512), (1024, 1024), (2048, 1024)),
                     steps_lo: int = 10_000, steps_hi: int = 500_000) -> list[dict]:
    """Poisson arrivals of melting runs: exponential gaps at ``rate_per_s``, grid
    drawn from ``grids``, step count log-uniform in [steps_lo, steps_hi], mixed
    parameters as in ``batch_draws``."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        nx, ny = grids[int(rng.integers(0, len(grids)))]
        p = cavity(nx, ny=ny,
                   porosity=float(rng.uniform(0.85, 0.98)),
                   Da=float(10 ** rng.uniform(-5, -3)),
                   Ra=float(10 ** rng.uniform(4, 6)),
                   Ste=float(rng.uniform(0.5, 2.0)))
        steps = int(round(10 ** rng.uniform(np.log10(steps_lo), np.log10(steps_hi))))
        out.append(dict(arrival_s=t, params=p, steps=steps))
    return out


def random_state(nx: int, ny: int, qt: int, seed: int, H_range=(0.0, 1.0), Tm_range=(0.0, 1.0),
                 rho_amp: float = 0.02, u_amp: float = 0.02, dT_amp: float = 0.01, f_base=None):
    """Random distributions for parity tests: arrays [q][ny][nx] (float64).

    Flow populations are positive values near ``f_base`` (9 values; 1/9 each
    by default) with relative noise; PCM
    populations are spread so that their sums land anywhere in ``H_range``;
    metal populations so that their sums land in ``Tm_range``; the exchange
    history is uniform noise of size ``dT_amp``."""
    rng = np.random.default_rng(seed)
    base = np.full(9, 1.0 / 9.0) if f_base is None else np.asarray(f_base, float).reshape(9)
    F = base[:, None, None] * (1.0 + rho_amp * rng.uniform(-1, 1, (9, ny, nx)))
    F[1:5] *= 1.0 + u_amp * rng.uniform(-1, 1, (4, ny, nx))
    Ht = rng.uniform(H_range[0], H_range[1], (ny, nx))
    G = np.empty((qt, ny, nx))
    share = rng.uniform(0.5, 1.5, (qt, ny, nx))
    share /= share.sum(axis=0, keepdims=True)
    G[...] = share * Ht[None]
    Tt = rng.uniform(Tm_range[0], Tm_range[1], (ny, nx))
    share = rng.uniform(0.5, 1.5, (qt, ny, nx))
    share /= share.sum(axis=0, keepdims=True)
    Hm = share * Tt[None]
    dT = dT_amp * rng.uniform(-1, 1, (ny, nx))
    return F, G, Hm, dT
