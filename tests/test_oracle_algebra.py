"""Pins of the oracle's single formulas against facts the paper and the
mathematics fix: lattice symmetry (Eq. 11), orthogonality of the transforms
(Eqs. 13, B1), consistency of each velocity-space equilibrium with its
moment-space counterpart (Eqs. 27/18, 40/34, 49/45, B3/B2, B5/B4), the forcing
moments against the velocity-space forcing of Guo and Zhao (ref. 74), the
explicit velocity root (Eqs. 22-25) and the enthalpy relations (Eqs. 29-30,
38-39)."""
import math

import numpy as np
import pytest

from paper_1701_00702_gb300 import inputs


def _params(qt=9, **over):
    p = inputs.cavity(16, thermal_q=qt)
    p.update(over)
    return p


def test_lattice_vectors_and_weights(oracle_mod):
    ex, ey, w = oracle_mod.lattice()
    assert list(ex) == [0, 1, 0, -1, 0, 1, -1, -1, 1]
    assert list(ey) == [0, 0, 1, 0, -1, 1, 1, -1, -1]
    assert abs(w.sum() - 1.0) < 1e-15
    # second moments of the weights give c_s^2 = 1/3 (Eq. 26); odd moments vanish
    assert abs((w * ex * ex).sum() - 1.0 / 3.0) < 1e-15
    assert abs((w * ey * ey).sum() - 1.0 / 3.0) < 1e-15
    assert abs((w * ex * ey).sum()) < 1e-15
    assert abs((w * ex).sum()) < 1e-15
    # fourth-order isotropy: sum w ex^4 = 3 sum w ex^2 ey^2 = 1/3
    assert abs((w * ex ** 4).sum() - 1.0 / 3.0) < 1e-15
    assert abs((w * ex ** 2 * ey ** 2).sum() - 1.0 / 9.0) < 1e-15


def test_d2q9_transform_inverse(oracle_mod):
    M, Mi = oracle_mod.matrices(9)
    assert np.abs(M @ Mi - np.eye(9)).max() < 1e-14
    # rows of Eq. 13 are orthogonal, so M^-1 = M^T diag(1/|row|^2)
    norms = np.array([9, 36, 36, 6, 12, 6, 12, 4, 4], float)
    assert np.allclose((M * M).sum(axis=1), norms, atol=0)
    assert np.abs(Mi - M.T / norms[None, :]).max() < 1e-15
    # the rows are the moments they are named for (Eq. 17): m3 = j_x, m5 = j_y
    ex, ey, _ = oracle_mod.lattice()
    assert np.array_equal(M[3], ex) and np.array_equal(M[5], ey)


def test_d2q5_transform_inverse(oracle_mod):
    M, Mi = oracle_mod.matrices(5)
    assert np.abs(M @ Mi - np.eye(5)).max() < 1e-15
    n = np.array([0.7, -0.2, 0.3, 1.1, 0.4])
    g = Mi @ n
    # closed-form inverse of Eq. B1
    expect = [n[0] - n[3], n[1] / 2 + (n[3] + n[4]) / 4, n[2] / 2 + (n[3] - n[4]) / 4,
              -n[1] / 2 + (n[3] + n[4]) / 4, -n[2] / 2 + (n[3] - n[4]) / 4]
    assert np.abs(g - expect).max() < 1e-15


@pytest.mark.parametrize("phi", [0.8, 0.9, 0.97])
def test_flow_equilibrium_moments(oracle_mod, phi):
    """Eq. 27 (velocity space) and Eq. 18 with alpha_1 = 1, alpha_2 = -3 describe
    the same equilibrium."""
    p = _params(porosity=phi)
    M, _ = oracle_mod.matrices(9)
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = 1.0 + 0.2 * rng.uniform(-1, 1)
        ux, uy = 0.1 * rng.uniform(-1, 1, 2)
        feq = oracle_mod.f_eq(p, rho, ux, uy)
        assert np.abs(M @ feq - oracle_mod.m_eq(p, rho, ux, uy)).max() < 1e-14


def test_forcing_moments_match_velocity_space_forcing(oracle_mod):
    """Eq. 19 equals M applied to the porous-medium forcing of Guo and Zhao
    (ref. 74): F_i = w_i rho [e.F/cs2 + ((e.u)(e.F) - cs2 u.F)/(phi cs2^2)]."""
    p = _params(porosity=0.85)
    M, _ = oracle_mod.matrices(9)
    ex, ey, w = oracle_mod.lattice()
    cs2 = 1.0 / 3.0
    rng = np.random.default_rng(2)
    for _ in range(20):
        rho = 1.0 + 0.1 * rng.uniform(-1, 1)
        ux, uy, Fx, Fy = 0.05 * rng.normal(size=4)
        eu, eF = ex * ux + ey * uy, ex * Fx + ey * Fy
        Fv = w * rho * (eF / cs2 + (eu * eF - cs2 * (ux * Fx + uy * Fy)) / (p["porosity"] * cs2 * cs2))
        assert np.abs(M @ Fv - oracle_mod.force_moments(p, rho, ux, uy, Fx, Fy)).max() < 1e-15


@pytest.mark.parametrize("qt", [5, 9])
def test_thermal_equilibrium_moments(oracle_mod, qt):
    """Eq. 40 vs Eq. 34 and Eq. 49 vs Eq. 45 (D2Q9); Eq. B3 vs B2 and B5 vs B4 (D2Q5)."""
    p = _params(qt=qt, porosity=0.9, cfref_over_cpl=0.3, cmref_over_cpm=0.8)
    M, _ = oracle_mod.matrices(qt)
    rng = np.random.default_rng(3)
    for _ in range(20):
        H, T, Tm = rng.uniform(-1, 3, 3)
        ux, uy = 0.1 * rng.uniform(-1, 1, 2)
        geq = oracle_mod.g_eq(p, H, T, ux, uy)
        assert abs(geq.sum() - H) < 1e-14                       # Eq. 37
        assert np.abs(M @ geq - oracle_mod.ng_eq(p, H, T, ux, uy)).max() < 1e-14
        heq = oracle_mod.h_eq(p, Tm)
        assert abs(heq.sum() - Tm) < 1e-14                      # Eq. 48 with c_pm = 1
        assert np.abs(M @ heq - oracle_mod.nh_eq(p, Tm)).max() < 1e-14


def test_velocity_root_solves_momentum_definition(oracle_mod):
    """Eq. 23 is the exact root of Eq. 22, u = (sum e f)/rho + F(u)/2 with F from Eq. 3."""
    rng = np.random.default_rng(4)
    for F_phi in (0.0, 0.068, 2.0):
        p = _params(porosity=0.8, Da=1e-3, F_phi=F_phi)
        lc = oracle_mod.lattice_config(p)
        for _ in range(20):
            rho = 1.0 + 0.1 * rng.uniform(-1, 1)
            jx, jy = 0.05 * rng.normal(size=2)
            Gy = 1e-3 * rng.normal()
            u = oracle_mod.velocity(p, rho, jx, jy, Gy)
            um = math.hypot(*u)
            phi, K = lc["phi"], lc["K"]
            F = -phi * lc["nu_f"] / K * u - phi * F_phi / math.sqrt(K) * um * u + phi * np.array([0.0, Gy])
            res = rho * u - (np.array([jx, jy]) + 0.5 * rho * F)
            assert np.abs(res).max() < 1e-15


def test_enthalpy_state_relations(oracle_mod):
    """Eqs. 38-39 satisfy Eqs. 29-30 (H = c_pf T + f_l L_a with c_pl = c_ps),
    are continuous at H_fs and H_fl, and H(T) inverts T(H) outside the mushy
    plateau."""
    for Ts, Tl, Ste in ((0.299, 0.301, 1.0), (-0.05, 0.05, 4.0), (0.0, 0.0, 1.0)):
        p = _params(T_solidus=Ts, T_liquidus=Tl, Ste=Ste)
        lc = oracle_mod.lattice_config(p)
        La = lc["L_a"]
        Hfs, Hfl = Ts, Tl + La
        for H in np.linspace(Hfs - 1.0, Hfl + 1.0, 301):
            T = oracle_mod.T_of_H(p, H)
            fl = oracle_mod.fl_of_H(p, H)
            assert 0.0 <= fl <= 1.0
            assert abs(T + fl * La - H) < 1e-13
        eps = 1e-12
        for Hb in (Hfs, Hfl):
            assert abs(oracle_mod.T_of_H(p, Hb - eps) - oracle_mod.T_of_H(p, Hb + eps)) < 1e-9
            assert abs(oracle_mod.fl_of_H(p, Hb - eps) - oracle_mod.fl_of_H(p, Hb + eps)) < 1e-9
        for T in (Ts - 0.5, Tl + 0.5):
            assert abs(oracle_mod.T_of_H(p, oracle_mod.H_of_T(p, T)) - T) < 1e-14


def test_relaxation_rates_follow_section_IIIC(oracle_mod):
    """Sec. III C / Eq. 53 / App. B: the rate map and its free constants."""
    lc = oracle_mod.lattice_config(_params(qt=9))
    za, ea = lc["zeta_a"], lc["eta_a"]
    assert lc["s"][:7] == [1.0, 1.1, 1.1, 1.0, 1.2, 1.0, 1.2]
    assert abs((1 / lc["s"][7] - 0.5) / 3.0 - lc["nu_e"]) < 1e-15               # Eq. 26
    assert abs((1 / lc["zeta"][1] - 0.5) * (1 / za - 0.5) - 0.25) < 1e-12        # Eq. 53
    assert abs((1 / za - 0.5) / 3.0 - lc["alpha_fref"]) < 1e-15                 # Eq. A19
    assert abs((1 / ea - 0.5) / 3.0 - lc["alpha_mref"]) < 1e-15                 # after Eq. 51
    assert lc["eta"] == [1.0, 1.1, 1.1, ea, ea, ea, ea, 1.2, 1.2]
    lc5 = oracle_mod.lattice_config(_params(qt=5, varpi=0.5))
    assert abs(lc5["csT2"] - 0.25) < 1e-15                                       # c_sT^2 = varpi/2
    assert abs((1 / lc5["zeta_a"] - 0.5) * 0.25 - lc5["alpha_fref"]) < 1e-15
