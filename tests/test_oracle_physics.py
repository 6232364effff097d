"""Pins of the oracle's full time step against what the macroscopic model and
exact invariants fix: conservation in a periodic box, zero velocity in solid
nodes, diffusion rates of both thermal lattices (Eq. 50-51, A19), the
interstitial exchange with its time-derivative correction (Eqs. 36, 47,
Remark III), the one-phase Stefan problem and its local-thermal-equilibrium
limit (Eqs. 28, 41, 10), the Brinkman-Forchheimer channel (Eqs. 2-3), a
decaying shear wave (Eq. 26 and the Darcy term of Eq. 3), adiabatic walls
(Eq. 52), a two-step hand calculation of the D2Q5 enthalpy update
(Eqs. 38, 52, B1-B3), and the thickness of the cavity's interface region
(Sec. IV B)."""
import math

import numpy as np
import pytest

from paper_1701_00702_gb300 import inputs
from tests import analytic


def _equilibrium_state(oracle_mod, p, T_f, T_m, ux=None, uy=None, rho=None):
    """Node-wise equilibrium distributions for given fields (uses the oracle's
    own equilibria, which test_oracle_algebra pins)."""
    lc = oracle_mod.lattice_config(p)
    ny, nx = T_f.shape
    qt = lc["qt"]
    F = np.zeros((9, ny, nx))
    G = np.zeros((qt, ny, nx))
    Hm = np.zeros((qt, ny, nx))
    for j in range(ny):
        for i in range(nx):
            u0 = 0.0 if ux is None else ux[j, i]
            u1 = 0.0 if uy is None else uy[j, i]
            r = 1.0 if rho is None else rho[j, i]
            F[:, j, i] = oracle_mod.f_eq(p, r, u0, u1)
            G[:, j, i] = oracle_mod.g_eq(p, oracle_mod.H_of_T(p, T_f[j, i]), T_f[j, i], u0, u1)
            Hm[:, j, i] = oracle_mod.h_eq(p, T_m[j, i])
    return F, G, Hm


@pytest.mark.parametrize("qt", [5, 9])
def test_mass_and_enthalpy_conserved_in_periodic_box(oracle_mod, qt):
    """Sum rho is kept by the blend (Eq. 20) and the collision (m_0); the total
    enthalpy sum[phi rho_l H_f + (1-phi) rho_m c_pm T_m] is kept because the two
    exchange sources (Eqs. 36, 47) cancel, time-derivative terms included."""
    p = inputs.periodic_box(24, 20, thermal_q=qt, Ra=1e7)
    o = oracle_mod.Oracle(p)
    assert 0.0 < o.lc["h_v"]
    F, G, Hm, dT = inputs.random_state(24, 20, qt, seed=11, H_range=(0.2, 1.4), Tm_range=(0.0, 1.0))
    o.set_state(F, G, Hm, dT)
    d0 = o.diag()
    o.run(300)
    d1 = o.diag()
    assert abs(d1["mass"] / d0["mass"] - 1.0) < 1e-13
    assert abs(d1["enthalpy"] / d0["enthalpy"] - 1.0) < 1e-12
    f = o.fields()
    assert np.isfinite(f["u_x"]).all() and np.abs(f["u_x"]).max() > 0.0


def test_solid_nodes_have_zero_velocity(oracle_mod):
    """f_l = 0 gives f = f^eq(rho, 0) (Eq. 20) and G = 0 (Eq. 7), hence u = 0 exactly."""
    p = inputs.periodic_box(16, 12, thermal_q=5)
    o = oracle_mod.Oracle(p)
    F, G, Hm, dT = inputs.random_state(16, 12, 5, seed=12, H_range=(-0.5, 0.9), Tm_range=(0.0, 1.0))
    o.set_state(F, G, Hm, dT)
    for _ in range(3):
        f = o.fields()
        solid = f["f_l"] == 0.0
        assert solid.sum() > 10
        assert np.all(f["u_x"][solid] == 0.0) and np.all(f["u_y"][solid] == 0.0)
        assert np.abs(f["u_x"][~solid]).max() > 0.0
        o.run(5)


def _decay_errors(oracle_mod, N, qt):
    p = inputs.periodic_box(N, 1, flow=0, thermal_q=qt, Nu_i=0.0, T_init=1.0, k_f=0.02,
                            cfref_over_cpl=0.5, cond_ratio=2.0, L_char=N)
    o = oracle_mod.Oracle(p)
    lc = o.lc
    k = 2.0 * math.pi / N
    T = 1.0 + 0.1 * np.sin(k * np.arange(N))[None, :]
    F, G, Hm = _equilibrium_state(oracle_mod, p, T, T)
    o.set_state(F, G, Hm, np.zeros((1, N)))
    o.run(50)
    f1 = o.fields()
    o.run(400)
    f2 = o.fields()
    rf = -math.log(analytic.mode_amplitude(f2["T_f"][0], k) / analytic.mode_amplitude(f1["T_f"][0], k)) / 400
    rm = -math.log(analytic.mode_amplitude(f2["T_m"][0], k) / analytic.mode_amplitude(f1["T_m"][0], k)) / 400
    ef = lc["alpha_fref"] * lc["c_fref"] * k * k / lc["c_pl"]   # Eq. 50 with u = 0, all liquid
    em = lc["alpha_mref"] * lc["c_mref"] * k * k / lc["c_pm"]   # Eq. 51
    return rf / ef - 1.0, rm / em - 1.0


@pytest.mark.parametrize("qt", [5, 9])
def test_thermal_diffusion_rates_converge_second_order(oracle_mod, qt):
    e32 = _decay_errors(oracle_mod, 32, qt)
    e64 = _decay_errors(oracle_mod, 64, qt)
    for a, b in zip(e32, e64):
        assert abs(b) < 1e-3
        assert 3.5 < a / b < 4.5


@pytest.mark.parametrize("qt", [5, 9])
def test_interstitial_exchange_is_adams_bashforth(oracle_mod, qt):
    """Uniform fields: summing Eq. 31 over i gives H(t+1) = H(t) + 1.5 Sr(t) - 0.5 Sr(t-1)
    (Eq. 36 with the backward difference of Remark III); likewise for T_m.
    The gap T_m - T_f then follows exp(-lambda t), lambda = h_v [1/(phi rho_l) + 1/((1-phi) rho_m)]."""
    p = inputs.periodic_box(4, 3, flow=0, thermal_q=qt, Nu_i=0.41, T_init=1.0, k_f=0.02,
                            porosity=0.9, L_char=100.0)
    o = oracle_mod.Oracle(p)
    lc = o.lc
    Tf0, Tm0 = 1.0, 1.5
    F, G, Hm = _equilibrium_state(oracle_mod, p, np.full((3, 4), Tf0), np.full((3, 4), Tm0))
    o.set_state(F, G, Hm, np.full((3, 4), Tm0 - Tf0))
    a_f = lc["h_v"] / (lc["phi"] * lc["rho_l"])
    a_m = lc["h_v"] / ((1.0 - lc["phi"]) * lc["rho_m"])
    lam = a_f + a_m
    assert 0.04 < lam < 0.06
    H, Tm, prev = oracle_mod.H_of_T(p, Tf0), Tm0, Tm0 - Tf0
    n = 100
    for _ in range(n):
        d = Tm - (H - lc["L_a"])          # all liquid: T_f = H - L_a
        H += a_f * (1.5 * d - 0.5 * prev)
        Tm -= a_m * (1.5 * d - 0.5 * prev)
        prev = d
    o.run(n)
    f = o.fields()
    assert np.abs(f["H_f"] - H).max() < 1e-13
    assert np.abs(f["T_m"] - Tm).max() < 1e-13
    gap = float(f["T_m"][0, 0] - f["T_f"][0, 0])
    assert abs(gap / ((Tm0 - Tf0) * math.exp(-lam * n)) - 1.0) < 1e-2


@pytest.mark.parametrize("qt", [5, 9])
def test_stefan_front_pcm_alone(oracle_mod, qt):
    """H_v = 0 decouples the lattices.  PCM: one-phase Neumann solution
    s = 2 kappa sqrt(alpha_f t), T_f = 1 - erf(x/2 sqrt(alpha_f t))/erf(kappa);
    metal: T_m = erfc(x / 2 sqrt(alpha_m t))."""
    from scipy.special import erf, erfc
    nx, n = 600, 20000
    p = inputs.conduction_1d(nx=nx, ny=1, thermal_q=qt, Nu_i=0.0, cond_ratio=10.0, L_char=100.0)
    o = oracle_mod.Oracle(p).run(n)
    lc = o.lc
    f = o.fields()
    kap = analytic.stefan_kappa(p["Ste"])
    a_f = lc["k_f"] / (lc["rho_l"] * lc["c_pl"])
    a_m = lc["k_m"] / (lc["rho_m"] * lc["c_pm"])
    s_exact = 2.0 * kap * math.sqrt(a_f * n)
    s_lb = f["f_l"][0].sum() - 0.5     # the wall node holds half a cell
    assert abs(s_lb - s_exact) < 1.0
    x = np.arange(nx, dtype=float)
    liquid = x < s_exact - 2.0
    T_exact = 1.0 - erf(x / (2.0 * math.sqrt(a_f * n))) / math.erf(kap)
    assert np.abs(f["T_f"][0][liquid] - T_exact[liquid]).max() < 1e-2
    assert np.abs(f["T_m"][0] - erfc(x / (2.0 * math.sqrt(a_m * n)))).max() < 1e-4


def test_stefan_front_lte_limit(oracle_mod):
    """Fast interstitial exchange: both phases share one temperature and the front
    follows the Neumann solution of Eq. 10 with k_e = phi k_f + (1-phi) k_m,
    (rho c)_e = phi rho_l c_pl + (1-phi) rho_m c_pm and latent heat phi rho_l L_a."""
    nx, n = 600, 20000
    p = inputs.conduction_1d(nx=nx, ny=1, thermal_q=5, Nu_i=4.33, cond_ratio=10.0, L_char=500.0)
    o = oracle_mod.Oracle(p).run(n)
    lc = o.lc
    phi = lc["phi"]
    k_e = phi * lc["k_f"] + (1 - phi) * lc["k_m"]
    rc = phi * lc["rho_l"] * lc["c_pl"] + (1 - phi) * lc["rho_m"] * lc["c_pm"]
    St_eff = rc * lc["dT"] / (phi * lc["rho_l"] * lc["L_a"])
    s_exact = 2.0 * analytic.stefan_kappa(St_eff) * math.sqrt(k_e / rc * n)
    s_lb = o.fields()["f_l"][0].sum() - 0.5
    assert abs(s_lb / s_exact - 1.0) < 1e-2


def test_adiabatic_walls_keep_one_dimensional_solution(oracle_mod):
    """Adiabatic top/bottom walls (Eq. 52 with T_b = T(x_f)) reproduce the
    y-periodic one-dimensional run exactly."""
    n = 300
    per = oracle_mod.Oracle(inputs.conduction_1d(nx=40, ny=1, Nu_i=1.0, L_char=100.0)).run(n).fields()
    wal = oracle_mod.Oracle(inputs.conduction_1d(nx=40, ny=5, Nu_i=1.0, periodic_y=0, L_char=100.0)).run(n).fields()
    for key in ("T_f", "T_m", "f_l", "H_f"):
        assert np.abs(wal[key] - per[key][0][None, :]).max() < 1e-14, key


def _channel(oracle_mod, nx, L, steps, Ra, F_phi):
    p = inputs.cavity(nx, ny=1, periodic_y=1, wall_kind=[0, 0, 1, 1], wall_T=[1.0, 1.0, 0.0, 0.0],
                      T_init=1.0, k_f=0.02, Pr=5.0, Da=0.04, Ra=Ra, L_char=L, F_phi=F_phi,
                      Nu_i=0.0, porosity=0.9)
    o = oracle_mod.Oracle(p).run(steps)
    lc = o.lc
    u = o.fields()["u_y"][0]
    G = lc["gbeta"] * (1.0 - lc["T0"])
    H = nx - 1
    if F_phi == 0.0:
        ref = analytic.brinkman_channel(np.arange(nx, dtype=float), H, G, lc["K"], lc["nu_f"], lc["nu_e"], lc["phi"])
    else:
        ref = analytic.forchheimer_channel_fd(H, G, lc["K"], lc["nu_f"], lc["nu_e"], lc["phi"], F_phi)
    return float(np.sqrt(((u - ref) ** 2).sum() / (ref ** 2).sum()))


def test_brinkman_channel_profile(oracle_mod):
    """Steady Eq. 2-3 between no-slip walls (non-equilibrium extrapolation, u_b = 0)
    driven by a uniform buoyancy G (uniform liquid temperature, Eq. 7)."""
    e17 = _channel(oracle_mod, 17, 16.0, 6000, 786.0, 0.0)
    e33 = _channel(oracle_mod, 33, 32.0, 12000, 393.0, 0.0)
    assert e33 < 3e-3
    assert e17 / e33 > 3.0


def test_forchheimer_channel_profile(oracle_mod):
    """Same channel with a strong Forchheimer term (F_phi = 3), against a fine
    finite-difference solution; the Forchheimer drag lowers the peak by ~40%."""
    e33 = _channel(oracle_mod, 33, 32.0, 12000, 393.0, 3.0)
    e65 = _channel(oracle_mod, 65, 64.0, 40000, 393.0 / 8.0, 3.0)
    assert e33 < 4e-3
    assert e65 < 1.2e-3


def _shear_error(oracle_mod, N, Da):
    p = inputs.periodic_box(4, N, flow=1, thermal_q=5, Nu_i=0.0, T_init=1.0, T_ref0=1.0, k_f=0.02,
                            Pr=5.0, Da=Da, L_char=32.0, F_phi=0.0, porosity=0.9)
    o = oracle_mod.Oracle(p)
    lc = o.lc
    k = 2.0 * math.pi / N
    ux = 1e-4 * np.sin(k * np.arange(N))[:, None] * np.ones((1, 4))
    F, G, Hm = _equilibrium_state(oracle_mod, p, np.ones((N, 4)), np.ones((N, 4)), ux=ux)
    o.set_state(F, G, Hm, np.zeros((N, 4)))
    o.run(20)
    a1 = analytic.mode_amplitude(o.fields()["u_x"][:, 0], k)
    o.run(200)
    a2 = analytic.mode_amplitude(o.fields()["u_x"][:, 0], k)
    rate = -math.log(a2 / a1) / 200
    return rate / (lc["nu_e"] * k * k + lc["phi"] * lc["nu_f"] / lc["K"]) - 1.0


def test_shear_wave_decay(oracle_mod):
    """A shear wave decays at nu_e k^2 + phi nu_f / K (Eq. 2-3 linearised; the
    advection term vanishes for a shear wave)."""
    e32 = _shear_error(oracle_mod, 32, 1e9)
    e64 = _shear_error(oracle_mod, 64, 1e9)
    assert abs(e64) < 1e-3 and 3.5 < e32 / e64 < 4.5
    assert abs(_shear_error(oracle_mod, 32, 0.04)) < 1e-3


def test_two_step_hand_calculation_d2q5(oracle_mod):
    """Hot Dirichlet wall (T_b = 1, H_b = 2) against PCM at its melting point
    (T_fs = T_fl = 0, H = 0, all g = 0), no exchange.  By hand from Eqs. 52,
    B1-B3: after step 1 node x=1 holds g_1 = a with a = varpi c_fref T_b / 4; its
    collision gives n* = (a, a(1-z_a), 0, a(1-z_e), a(1-z_eps)), so the g_1 it
    sends to x=2 is a(2 - z_a - z_eps)/4 with z_e = 2 - z_a.  That value is the
    enthalpy of x=2 after step 2; it is negative because z_a > 1 over-relaxes
    the flux moment."""
    p = inputs.conduction_1d(nx=12, ny=1, thermal_q=5, Nu_i=0.0)
    o = oracle_mod.Oracle(p)
    lc = o.lc
    a = lc["varpi"] * lc["c_fref"] * 1.0 / 4.0
    o.run(1)
    H1 = o.fields()["H_f"][0]
    assert abs(H1[1] - a) < 1e-15 and np.all(H1[2:-1] == 0.0)
    o.run(1)
    H2 = o.fields()["H_f"][0]
    expect = a * (2.0 - lc["zeta_a"] - lc["zeta"][4]) / 4.0
    assert abs(H2[2] - expect) < 1e-15
    assert expect < 0.0


@pytest.mark.parametrize("qt", [5, 9])
def test_temperature_mode_advects_at_u_over_phi(oracle_mod, qt):
    """A uniform flow U (no drag: Da huge, F_phi = 0; no buoyancy: Ra = 0) carries
    a temperature mode at U/phi, the convective speed of Eq. 28 with H = T + L_a."""
    N, U = 64, 0.02
    p = inputs.periodic_box(N, 1, flow=1, thermal_q=qt, Nu_i=0.0, T_init=1.0, k_f=0.01, Pr=1.0,
                            Ra=0.0, Da=1e9, F_phi=0.0, L_char=N, porosity=0.8, cfref_over_cpl=0.5)
    o = oracle_mod.Oracle(p)
    k = 2.0 * math.pi / N
    x = np.arange(N)
    T = 1.0 + 0.1 * np.sin(k * x)[None, :]
    F, G, Hm = _equilibrium_state(oracle_mod, p, T, T, ux=np.full((1, N), U))
    o.set_state(F, G, Hm, np.zeros((1, N)))

    def phase(v):
        w = v - v.mean()
        return math.atan2(float((w * np.cos(k * x)).sum()), float((w * np.sin(k * x)).sum()))

    o.run(10)
    p1 = phase(o.fields()["T_f"][0])
    o.run(200)
    f = o.fields()
    speed = -(phase(f["T_f"][0]) - p1) / (k * 200)
    assert abs(speed / (U / o.lc["phi"]) - 1.0) < 2e-3
    assert abs(f["u_x"].mean() / U - 1.0) < 1e-9


@pytest.mark.parametrize("qt", [5, 9])
def test_coupled_two_temperature_mode(oracle_mod, qt):
    """Sine modes of T_f and T_m with interstitial exchange follow the 2x2 linear
    system of Eqs. 28 and 41 (u = 0, all liquid):
    d/dt [T_f, T_m] = [[-D_f k^2 - a_f, a_f], [a_m, -D_m k^2 - a_m]] [T_f, T_m]
    with D = alpha_ref c_ref, a_f = h_v/(phi rho_l), a_m = h_v/((1-phi) rho_m);
    second-order convergence in the grid."""
    from scipy.linalg import expm
    errs = []
    for N in (32, 64):
        p = inputs.periodic_box(N, 1, flow=0, thermal_q=qt, Nu_i=0.41, T_init=1.0, k_f=0.02,
                                porosity=0.9, cond_ratio=3.0, L_char=100.0, cfref_over_cpl=0.5)
        o = oracle_mod.Oracle(p)
        lc = o.lc
        k = 2.0 * math.pi / N
        x = np.arange(N)
        Tf = 1.0 + 0.1 * np.sin(k * x)[None, :]
        Tm = 1.0 + 0.05 * np.sin(k * x)[None, :]
        F, G, Hm = _equilibrium_state(oracle_mod, p, Tf, Tm)
        o.set_state(F, G, Hm, Tm - Tf)
        a_f = lc["h_v"] / (lc["phi"] * lc["rho_l"])
        a_m = lc["h_v"] / ((1.0 - lc["phi"]) * lc["rho_m"])
        D_f = lc["alpha_fref"] * lc["c_fref"]
        D_m = lc["alpha_mref"] * lc["c_mref"]
        A = np.array([[-D_f * k * k - a_f, a_f], [a_m, -D_m * k * k - a_m]])
        n = 300
        o.run(n)
        f = o.fields()
        ref = expm(A * n) @ np.array([0.1, 0.05])
        got = np.array([2.0 / N * float(((v[0] - v[0].mean()) * np.sin(k * x)).sum()) for v in (f["T_f"], f["T_m"])])
        errs.append(np.abs(got / ref - 1.0).max())
    assert errs[1] < 1e-3
    assert 3.5 < errs[0] / errs[1] < 5.0


def test_shear_wave_is_advected_at_u_over_phi(oracle_mod):
    """A shear wave u_x(y) riding on a uniform u_y = U travels at U/phi: the
    convective term (u.grad)(u/phi) of Eq. 2 carried by the porous equilibrium
    moments (Eq. 18)."""
    N, U = 64, 0.02
    p = inputs.periodic_box(4, N, flow=1, thermal_q=5, Nu_i=0.0, T_init=1.0, T_ref0=1.0, k_f=0.02,
                            Pr=5.0, Da=1e9, L_char=32.0, F_phi=0.0, porosity=0.8)
    o = oracle_mod.Oracle(p)
    k = 2.0 * math.pi / N
    y = np.arange(N)
    ux = 1e-3 * np.sin(k * y)[:, None] * np.ones((1, 4))
    F, G, Hm = _equilibrium_state(oracle_mod, p, np.ones((N, 4)), np.ones((N, 4)), ux=ux, uy=np.full((N, 4), U))
    o.set_state(F, G, Hm, np.zeros((N, 4)))

    def phase(v):
        w = v - v.mean()
        return math.atan2(float((w * np.cos(k * y)).sum()), float((w * np.sin(k * y)).sum()))

    o.run(10)
    p1 = phase(o.fields()["u_x"][:, 0])
    o.run(200)
    d = -(phase(o.fields()["u_x"][:, 0]) - p1)
    d = (d + math.pi) % (2.0 * math.pi) - math.pi
    assert abs(d / (k * 200) / (U / o.lc["phi"]) - 1.0) < 1e-3


@pytest.mark.parametrize("qt", [5, 9])
def test_exchange_source_is_distributed_like_the_equilibrium(oracle_mod, qt):
    """The moment-space source directions (1,-2,1,0,...) of Eqs. 35/46 and
    (1,0,0,varpi,0) of App. B are M applied to the equilibrium weights, so with
    c_ref = c_p a uniform equilibrium state plus one exchange step is again an
    equilibrium: g* = g^eq(H + S_PCM, T(H + S_PCM)), h* = h^eq(T_m + S_metal/c_pm)."""
    p = inputs.periodic_box(3, 2, flow=0, thermal_q=qt, Nu_i=0.41, T_init=1.0, k_f=0.02,
                            porosity=0.9, L_char=100.0, cfref_over_cpl=1.0, cmref_over_cpm=1.0)
    o = oracle_mod.Oracle(p)
    lc = o.lc
    Tf0, Tm0 = 1.0, 1.4
    F, G, Hm = _equilibrium_state(oracle_mod, p, np.full((2, 3), Tf0), np.full((2, 3), Tm0))
    o.set_state(F, G, Hm, np.full((2, 3), Tm0 - Tf0))      # d/dt Sr = 0 at the start
    o.run(1)
    _, G1, H1, _ = o.state()
    S_f = lc["h_v"] * (Tm0 - Tf0) / (lc["phi"] * lc["rho_l"])
    S_m = -lc["h_v"] * (Tm0 - Tf0) / ((1.0 - lc["phi"]) * lc["rho_m"])
    H_new = oracle_mod.H_of_T(p, Tf0) + S_f
    g_expect = oracle_mod.g_eq(p, H_new, oracle_mod.T_of_H(p, H_new), 0.0, 0.0)
    h_expect = oracle_mod.h_eq(p, Tm0 + S_m / lc["c_pm"])
    assert np.abs(G1 - g_expect[:, None, None]).max() < 1e-15
    assert np.abs(H1 - h_expect[:, None, None]).max() < 1e-15


# ---- comparison variants of Sec. V ------------------------------------------

@pytest.mark.parametrize("qt", [5, 9])
def test_bgk_thermal_collision_keeps_the_diffusivity(oracle_mod, qt):
    """Sec. V A's BGK thermal lattices (every rate zeta_alpha, eta_alpha) recover
    the same diffusivities alpha_ref c_ref (Eq. A19 fixes them through zeta_alpha
    alone): decay rates converge at second order.  Their error is larger than
    with the MRT rates of Eq. 53 (1.1e-3 against 2e-4 at N = 64), the reduced
    numerical diffusion Sec. V A credits to MRT."""
    errs = []
    for N in (32, 64):
        p = inputs.periodic_box(N, 1, flow=0, thermal_q=qt, Nu_i=0.0, T_init=1.0, k_f=0.02,
                                cfref_over_cpl=0.5, cond_ratio=2.0, L_char=N, thermal_collision=1)
        lc = oracle_mod.lattice_config(p)
        assert lc["zeta"][:qt] == [lc["zeta_a"]] * qt and lc["eta"][:qt] == [lc["eta_a"]] * qt
        o = oracle_mod.Oracle(p)
        k = 2.0 * math.pi / N
        T = 1.0 + 0.1 * np.sin(k * np.arange(N))[None, :]
        F, G, Hm = _equilibrium_state(oracle_mod, p, T, T)
        o.set_state(F, G, Hm, np.zeros((1, N)))
        o.run(50)
        a1 = analytic.mode_amplitude(o.fields()["T_f"][0], k)
        o.run(400)
        a2 = analytic.mode_amplitude(o.fields()["T_f"][0], k)
        errs.append(-math.log(a2 / a1) / 400 / (lc["alpha_fref"] * lc["c_fref"] * k * k) - 1.0)
    assert abs(errs[1]) < 2e-3 and 3.5 < errs[0] / errs[1] < 4.5


@pytest.mark.parametrize("value", [1.8, 1.2, 0.6, 0.1])
def test_explicit_zeta_e_replaces_eq_53(oracle_mod, value):
    """Sec. V D sweeps zeta_e over 1.8, 1.2, 0.6, 0.1 instead of 2 - zeta_alpha."""
    p = inputs.paper_cavity_defaults()
    p.update(thermal_q=9, zeta_e=value)
    lc = oracle_mod.lattice_config(p)
    assert lc["zeta"][1] == lc["zeta"][2] == value
    p.update(thermal_q=5)
    assert oracle_mod.lattice_config(p)["zeta"][3] == value


def test_bounce_back_conserves_mass_and_stops_solid_nodes(oracle_mod):
    p = inputs.periodic_box(20, 16, thermal_q=5, Ra=1e7, solid_scheme=1)
    o = oracle_mod.Oracle(p)
    F, G, Hm, dT = inputs.random_state(20, 16, 5, seed=21, H_range=(-0.2, 1.6))
    o.set_state(F, G, Hm, dT)
    m0 = o.diag()["mass"]
    o.run(200)
    f = o.fields()
    assert abs(o.diag()["mass"] / m0 - 1.0) < 1e-13
    solid = f["f_l"] <= 0.5
    assert solid.sum() > 10 and (~solid).sum() > 10
    assert np.all(f["u_x"][solid] == 0.0) and np.all(f["u_y"][solid] == 0.0)


def test_bounce_back_channel_between_solid_layers(oracle_mod):
    """Sec. V B's bounce-back scheme: a liquid layer between solid columns
    (f_l = 0; liquid and solid held just above and below an isothermal melting
    point so the layers stay put) carries the Brinkman profile with the walls
    half-way between the last liquid and the first solid node."""
    errs = []
    for nf, steps in ((16, 4000), (32, 10000)):
        nx = nf + 4
        p = inputs.cavity(nx, ny=1, periodic_x=1, periodic_y=1, solid_scheme=1, Nu_i=0.0, k_f=1e-3, Pr=100.0,
                          Da=0.04, L_char=float(nf), T_solidus=0.3, T_liquidus=0.3, T_init=0.3, T_ref0=0.0,
                          Ra=393.0, porosity=0.9, F_phi=0.0)
        lc = oracle_mod.lattice_config(p)
        o = oracle_mod.Oracle(p)
        T = np.full((1, nx), 0.3)
        F, G, Hm = _equilibrium_state(oracle_mod, p, T, T)
        for x in range(nx):
            H = lc["T_fs"] - 0.01 if (x < 2 or x >= nx - 2) else lc["T_fl"] + lc["L_a"] + 0.01
            Tx = oracle_mod.T_of_H(p, H)
            G[:, 0, x] = oracle_mod.g_eq(p, H, Tx, 0.0, 0.0)
            Hm[:, 0, x] = oracle_mod.h_eq(p, Tx)
        o.set_state(F, G, Hm, np.zeros((1, nx)))
        o.run(steps)
        f = o.fields()
        assert f["f_l"][0][:2].max() <= 0.5 and f["f_l"][0][2:-2].min() == 1.0
        Gv = lc["gbeta"] * (f["T_f"][0, nx // 2] - lc["T0"])
        ref = analytic.brinkman_channel(np.arange(nx) - 1.5, float(nf), Gv, lc["K"], lc["nu_f"], lc["nu_e"], lc["phi"])
        u = f["u_y"][0]
        errs.append(float(np.sqrt(((u[2:-2] - ref[2:-2]) ** 2).sum() / (ref[2:-2] ** 2).sum())))
    assert errs[0] < 1e-2 and errs[1] < errs[0]


# ---- phase-dependent PCM properties (Eq. 9) ----------------------------------

@pytest.mark.parametrize("qt", [5, 9])
@pytest.mark.parametrize("phase", ["solid", "liquid"])
def test_eq9_conductivity_sets_the_decay_of_each_phase(oracle_mod, qt, phase):
    """With k_s = k_l/2 and c_ps = 1.5 c_pl, a temperature mode inside one
    phase decays at k k^2/c_p of that phase (Eq. 28 with Eq. 9): the per-node
    zeta_alpha of Eq. A19 carries k_s or k_l, and Eq. 38 carries c_ps or c_pl.
    Second-order convergence, as for the constant-property lattice."""
    T0 = 0.1 if phase == "solid" else 0.6          # below T_fs = 0.299 or above T_fl = 0.301
    errs = []
    for N in (32, 64):
        p = inputs.periodic_box(N, 1, flow=0, thermal_q=qt, Nu_i=0.0, T_init=T0, k_f=0.02,
                                cfref_over_cpl=0.5, cond_ratio=2.0, L_char=N, ks_over_kl=0.5, cps_over_cpl=1.5)
        lc = oracle_mod.lattice_config(p)
        assert lc["phase_k"] == 1 and lc["c_ps"] == 1.5 and lc["k_s"] == 0.01
        o = oracle_mod.Oracle(p)
        k = 2.0 * math.pi / N
        T = T0 + 0.05 * np.sin(k * np.arange(N))[None, :]
        F, G, Hm = _equilibrium_state(oracle_mod, p, T, T)
        o.set_state(F, G, Hm, np.zeros((1, N)))
        o.run(50)
        a1 = analytic.mode_amplitude(o.fields()["T_f"][0], k)
        o.run(400)
        f = o.fields()
        assert np.all(f["f_l"] == (0.0 if phase == "solid" else 1.0))
        a2 = analytic.mode_amplitude(f["T_f"][0], k)
        kc = (lc["k_s"] / lc["c_ps"]) if phase == "solid" else (lc["k_l"] / lc["c_pl"])
        errs.append(-math.log(a2 / a1) / 400 / (kc * k * k) - 1.0)
    assert abs(errs[1]) < 1e-3 and 3.5 < errs[0] / errs[1] < 4.5


@pytest.mark.parametrize("qt", [5, 9])
def test_eq9_two_phase_neumann_front(oracle_mod, qt):
    """Melting into a subcooled solid with k_s = 2 k_l and c_ps = 1.5 c_pl
    (H_v = 0, u = 0): the front follows the two-phase Neumann solution
    s = 2 lambda sqrt(alpha_l t), and both temperature profiles follow
    their erf / erfc forms."""
    from scipy.special import erf, erfc
    nx, n, Ti = 400, 40000, -0.3
    p = inputs.conduction_1d(nx=nx, ny=1, thermal_q=qt, Nu_i=0.0, cond_ratio=10.0, L_char=100.0,
                             T_init=Ti, wall_T=[1.0, Ti, 0.0, 0.0], ks_over_kl=2.0, cps_over_cpl=1.5)
    o = oracle_mod.Oracle(p).run(n)
    lc = o.lc
    f = o.fields()
    a_l = lc["k_l"] / (lc["rho_l"] * lc["c_pl"])
    a_s = lc["k_s"] / (lc["rho_l"] * lc["c_ps"])
    nu = math.sqrt(a_l / a_s)
    lam = analytic.neumann_two_phase(lc["c_pl"] * 1.0 / lc["L_a"], lc["c_ps"] * (0.0 - Ti) / lc["L_a"], nu)
    lam_one = analytic.stefan_kappa(lc["c_pl"] / lc["L_a"])
    s_exact = 2.0 * lam * math.sqrt(a_l * n)
    assert 2.0 * lam_one * math.sqrt(a_l * n) - s_exact > 4.0     # subcooling slows the front visibly
    s_lb = f["f_l"][0].sum() - 0.5
    assert abs(s_lb - s_exact) < 1.0
    x = np.arange(nx, dtype=float)
    liquid = x < s_exact - 2.0
    solid = x > s_exact + 2.0
    T_l = 1.0 - erf(x / (2.0 * math.sqrt(a_l * n))) / math.erf(lam)
    T_s = Ti + (0.0 - Ti) * erfc(x / (2.0 * math.sqrt(a_s * n))) / math.erfc(nu * lam)
    assert np.abs(f["T_f"][0][liquid] - T_l[liquid]).max() < 1e-2
    assert np.abs(f["T_f"][0][solid] - T_s[solid]).max() < 1e-2


def test_eq9_variant_conserves_mass_and_enthalpy(oracle_mod):
    p = inputs.periodic_box(24, 20, thermal_q=5, Ra=1e7, ks_over_kl=0.4, cps_over_cpl=1.3)
    o = oracle_mod.Oracle(p)
    F, G, Hm, dT = inputs.random_state(24, 20, 5, seed=13, H_range=(0.0, 1.6), Tm_range=(0.0, 1.0))
    o.set_state(F, G, Hm, dT)
    d0 = o.diag()
    o.run(300)
    d1 = o.diag()
    assert abs(d1["mass"] / d0["mass"] - 1.0) < 1e-12
    assert abs(d1["enthalpy"] / d0["enthalpy"] - 1.0) < 1e-12


def test_eq9_two_step_hand_calculation_d2q5(oracle_mod):
    """The two-step hand calculation above with k_s = 3 k_l: node x=1 collides
    at f_l = a/L_a (isothermal mushy zone), so by Eq. 9 its conductivity is
    k = f_l k_l + (1 - f_l) k_s, by Eq. A19 zeta_a' = 1/(1/2 + k/(c_fref c_sT^2))
    and by Eq. 53 zeta_e' = 2 - zeta_a'.  The g_1 it sends to x=2 is
    a(4 - zeta_e' - z_eps - 2 zeta_a')/4 = a(2 - zeta_a' - z_eps)/4."""
    p = inputs.conduction_1d(nx=12, ny=1, thermal_q=5, Nu_i=0.0, ks_over_kl=3.0)
    o = oracle_mod.Oracle(p)
    lc = o.lc
    a = lc["varpi"] * lc["c_fref"] * 1.0 / 4.0
    o.run(1)
    assert abs(o.fields()["H_f"][0][1] - a) < 1e-15
    o.run(1)
    fl1 = a / lc["L_a"]
    k = fl1 * lc["k_l"] + (1.0 - fl1) * lc["k_s"]
    za = 1.0 / (0.5 + k / (lc["rho_l"] * lc["c_fref"] * lc["csT2"]))
    ze = 2.0 - za
    expect = a * (4.0 - ze - lc["zeta"][4] - 2.0 * za) / 4.0
    assert abs(o.fields()["H_f"][0][2] - expect) < 1e-15
    assert abs(za - lc["zeta_a"]) > 0.1                  # the node's rate is not the liquid one


def test_cavity_interface_region_is_about_ten_lattices_thick(oracle_mod):
    """Sec. IV B cavity at Ra = 1e6 on 150 x 150 (the paper's own set-up) up to
    Fo = t alpha_f / L^2 = 0.001 (Eq. 54; 45,000 steps): while the PCM melts
    the phase interface is a region about ten lattices thick (the paper's
    reading of Fig. 6, Fo <= 0.002), f_l stays in [0, 1], and the flow inside
    the interface region (f_l < 0.5) is much weaker than in the liquid (the
    volumetric scheme's damping, Sec. V B).  Measured: 14 lattices with
    0.01 < f_l < 0.99 in every row, |u_y| 1.1e-6 against |u| 8.2e-5."""
    p = dict(inputs.paper_cavity_defaults(), precision=0)
    o = oracle_mod.Oracle(p)
    steps = int(round(0.001 * p["L_char"] ** 2 / p["k_f"]))
    assert steps == 45000
    o.run(steps)
    f = o.fields()
    fl = f["f_l"]
    assert fl.min() >= 0.0 and fl.max() <= 1.0
    band = ((fl > 0.01) & (fl < 0.99)).sum(axis=1)[5:-5]     # rows away from the adiabatic walls
    assert 5 <= band.min() and band.max() <= 20, (band.min(), band.max())
    liquid, weak = fl >= 0.999, (fl > 0.0) & (fl < 0.5)
    assert liquid.any() and weak.any()
    u_liquid = np.hypot(f["u_x"], f["u_y"])[liquid].max()
    assert np.abs(f["u_y"][weak]).max() < 0.1 * u_liquid
    assert np.all(f["u_x"][fl == 0.0] == 0.0) and np.all(f["u_y"][fl == 0.0] == 0.0)
