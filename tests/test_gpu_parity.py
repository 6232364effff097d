"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Tolerances:
  * FP64 storage: element-wise agreement to a few ulps of the largest value
    (1e-12 relative) after one step; relative L2 <= 1e-10 after 20k steps.
  * FP32 storage: one step from identical inputs agrees to 5e-6 of the
    array's scale (FP32 rounding of a few dozen operations); after long runs
    the fields T_f, T_s (= T_m), f_l and u agree in relative L2 to 1e-5, the
    bound the method's stated target sets for the FP32 path.
"""
import numpy as np
import pytest

from paper_1701_00702_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1701_00702_gb300 import build, lbm as mod
    build.build()
    return mod


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.sqrt((b * b).sum())
    return float(np.sqrt(((a - b) ** 2).sum()) / (den if den > 0 else 1.0))


W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]   # Eq. 27 weights


def _as_precision(arrs, prec):
    dt = np.float64 if prec == 0 else np.float32
    return [None if a is None else np.asarray(a).astype(dt) for a in arrs]


def _random_pair(lbm, oracle_mod, p, seed, f_base=None):
    """Solver and oracle holding the same (precision-rounded) random state."""
    lc = oracle_mod.lattice_config(p)
    H_lo, H_hi = lc["T_fs"] - 0.3, lc["T_fl"] + lc["L_a"] + 0.3
    F, G, Hm, dT = inputs.random_state(p["nx"], p["ny"], p["thermal_q"], seed, H_range=(H_lo, H_hi),
                                       Tm_range=(0.0, 1.0), f_base=f_base)
    Fd, G, Hm, dT = _as_precision([F - W9, G, Hm, dT], p["precision"])
    s = lbm.Solver(p)
    s.set_state(Fd if p["flow"] else None, G, Hm, dT)
    o = oracle_mod.Oracle(p)
    o.set_state(Fd.astype(np.float64) + W9, G.astype(np.float64), Hm.astype(np.float64), dT.astype(np.float64))
    return s, o


def _compare_states(s, o, prec, flow):
    f, g, h, dT = s.get_state()
    F, G, H, D = o.state()
    tol = 1e-12 if prec == 0 else 5e-6
    pairs = [(g, G, "g"), (h, H, "h"), (dT, D, "dT")] + ([(f, F - W9, "f - w")] if flow else [])
    for a, b, name in pairs:
        # dT = T_m - T_f is a difference of O(1) temperatures: measure it on that scale
        scale = max(np.abs(b).max(), 1.0 if name == "dT" else 1e-3)
        err = np.abs(a.astype(np.float64) - b).max() / scale
        assert err < tol, (name, err)


SHAPES = [
    # (nx, ny, periodic_x, periodic_y): several 128 x 2 blocks with ragged tails, tiny grids
    (131, 7, 0, 0), (131, 7, 1, 1), (130, 9, 0, 1), (3, 3, 0, 0), (1, 1, 1, 1), (5, 1, 0, 1), (257, 4, 1, 0),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("qt", [5, 9])
@pytest.mark.parametrize("flow", [1, 0])
@pytest.mark.parametrize("shape", SHAPES)
def test_steps_from_random_state(lbm, oracle_mod, prec, qt, flow, shape):
    nx, ny, px, py = shape
    p = inputs.cavity(max(nx, ny), ny=ny, precision=prec, thermal_q=qt, flow=flow, periodic_x=px,
                      periodic_y=py, L_char=100.0, Ra=1e7)
    p["nx"] = nx
    s, o = _random_pair(lbm, oracle_mod, p, seed=nx * 31 + ny)
    s.step(1)
    o.run(1)
    _compare_states(s, o, prec, flow)
    s.step(2)
    o.run(2)
    _compare_states(s, o, prec, flow)
    fs = s.fields(device=False)
    fo = o.fields()
    for name, key in (("T_f", "T_f"), ("T_s", "T_m"), ("f_l", "f_l"), ("u_x", "u_x"), ("u_y", "u_y"),
                      ("rho", "rho"), ("H_f", "H_f")):
        scale = max(np.abs(fo[key]).max(), 1e-3)
        tol = 1e-12 if prec == 0 else 5e-6
        assert np.abs(fs[name].astype(np.float64) - fo[key]).max() / scale < tol, name
    s.close()


@pytest.mark.parametrize("qt", [5, 9])
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_conduction_melting_20k_steps(lbm, oracle_mod, qt, prec, tol):
    """Conduction-only LTNE melting, 200 x 4, 20,000 steps (the Sec. IV A constants)."""
    p = inputs.conduction_1d(thermal_q=qt, precision=prec)
    s = lbm.Solver(p)
    s.step(20000)
    assert s.status() == 0
    o = oracle_mod.Oracle(p).run(20000)
    fs, fo = s.fields(device=False), o.fields()
    for name, key in (("T_f", "T_f"), ("T_s", "T_m"), ("f_l", "f_l")):
        assert rel_l2(fs[name], fo[key]) <= tol, name
    assert np.all(fs["u_x"] == 0) and np.all(fs["u_y"] == 0)
    d_s, d_o = s.diag(), o.diag()
    assert abs(d_s["melt_frac"] - d_o["melt_frac"]) <= (1e-12 if prec == 0 else 1e-5)
    s.close()


def test_cavity_256_fp32_parity(lbm, oracle_mod):
    """Square-cavity melting with natural convection, 256 x 256, FP32, 2,000 steps:
    T_f, T_s, f_l, u_x, u_y against the oracle in relative L2."""
    p = inputs.cavity(256, precision=1)
    s = lbm.Solver(p)
    s.step(2000)
    assert s.status() == 0
    o = oracle_mod.Oracle(p).run(2000)
    fs, fo = s.fields(device=False), o.fields()
    for name, key in (("T_f", "T_f"), ("T_s", "T_m"), ("f_l", "f_l"), ("u_x", "u_x"), ("u_y", "u_y")):
        assert rel_l2(fs[name], fo[key]) <= 1e-5, name
    assert np.abs(fo["u_y"]).max() > 1e-7      # the flow is really on
    d_s, d_o = s.diag(), o.diag()
    for k in ("melt_frac", "nu_hot", "enthalpy", "mass"):
        assert abs(d_s[k] / d_o[k] - 1.0) < 1e-5, k
    s.close()


def test_diagnostics_match_oracle_fp64(lbm, oracle_mod):
    p = inputs.cavity(96, ny=80, precision=0, thermal_q=9)
    s = lbm.Solver(p)
    s.step(300)
    o = oracle_mod.Oracle(p).run(300)
    d_s, d_o = s.diag(), o.diag()
    for k in ("melt_frac", "nu_hot", "enthalpy", "mass"):
        assert abs(d_s[k] / d_o[k] - 1.0) < 1e-12, k
    # equal states give bit-equal diagnostics
    assert s.diag() == d_s
    s.close()


def test_full_size_sampled_parity_2048(lbm, oracle_mod):
    """2048 x 2048 cavity in FP32, the benchmark's launch configuration: one step
    from a random state checked against the oracle at sampled nodes (all four
    edges and corners plus random interior nodes)."""
    n = 2048
    p = inputs.cavity(n, precision=1)
    lc = oracle_mod.lattice_config(p)
    F, G, Hm, dT = inputs.random_state(n, n, 5, seed=2048, H_range=(lc["T_fs"] - 0.3, lc["T_fl"] + lc["L_a"] + 0.3))
    Fd, G, Hm, dT = _as_precision([F - W9, G, Hm, dT], 1)
    del F
    s = lbm.Solver(p)
    s.set_state(Fd, G, Hm, dT)
    s.step(1)
    f1, g1, h1, d1 = s.get_state()
    o = oracle_mod.Oracle(p)
    o.set_state(Fd.astype(np.float64) + W9, G.astype(np.float64), Hm.astype(np.float64), dT.astype(np.float64))
    rng = np.random.default_rng(7)
    edge = np.arange(n)
    xs = np.concatenate([edge, edge, np.zeros(n, int), np.full(n, n - 1), rng.integers(0, n, 20000)])
    ys = np.concatenate([np.zeros(n, int), np.full(n, n - 1), edge, edge, rng.integers(0, n, 20000)])
    fo, go, ho, do = o.step_nodes(xs, ys)
    fo = fo - W9[:, 0, 0][None, :]
    for a, b, floor in ((f1[:, ys, xs].T, fo, 1e-3), (g1[:, ys, xs].T, go, 1e-3), (h1[:, ys, xs].T, ho, 1e-3),
                        (d1[ys, xs], do, 1.0)):
        assert np.abs(a.astype(np.float64) - b).max() / max(np.abs(b).max(), floor) < 5e-6
    s.close()


def test_full_size_invariants_2048(lbm):
    """Properties that hold at any size, on the benchmark's 2048 x 2048 FP32 cavity
    after 2,000 steps from the uniform start: finite, 0 <= f_l <= 1, u = 0 exactly
    in solid nodes and on walls, melting has started at the hot wall only."""
    s = lbm.Solver(inputs.cavity(2048, precision=1))
    s.step(2000)
    assert s.status() == 0
    f = s.fields(device=False)
    fl, ux, uy = f["f_l"], f["u_x"], f["u_y"]
    assert np.isfinite(f["T_f"]).all() and np.isfinite(ux).all()
    assert fl.min() >= 0.0 and fl.max() <= 1.0
    solid = fl == 0.0
    assert solid.mean() > 0.9
    assert np.all(ux[solid] == 0.0) and np.all(uy[solid] == 0.0)
    assert np.all(ux[:, 0] == 0) and np.all(uy[0, :] == 0) and np.all(ux[:, -1] == 0)
    assert fl[:, 1].mean() > 0.5 and fl[:, -2].max() == 0.0
    s.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-5)])
def test_periodic_box_conserves_mass_and_enthalpy(lbm, prec, tol):
    p = inputs.periodic_box(512, 384, precision=prec, Ra=1e7)
    F, G, Hm, dT = inputs.random_state(512, 384, 5, seed=5, H_range=(0.2, 1.4))
    Fd, G, Hm, dT = _as_precision([F - W9, G, Hm, dT], prec)
    s = lbm.Solver(p)
    s.set_state(Fd, G, Hm, dT)
    d0 = s.diag()
    s.step(500)
    d1 = s.diag()
    assert abs(d1["mass"] / d0["mass"] - 1) < tol
    assert abs(d1["enthalpy"] / d0["enthalpy"] - 1) < tol
    s.close()


def test_graph_replay_equals_single_launches(lbm):
    p = inputs.cavity(150, precision=1)
    a, b = lbm.Solver(p), lbm.Solver(p)
    a.step(3)
    a.step(130)          # odd start: single launches, then two captured 64-step graphs
    for _ in range(133):
        b.step(1)
    fa, fb = a.get_state(with_lo=True), b.get_state(with_lo=True)
    for x, y in zip(fa, fb):
        assert np.array_equal(x, y)
    assert a.steps == b.steps == 133
    a.close(); b.close()


def test_checkpoint_resume_is_bitwise(lbm):
    p = inputs.cavity(128, precision=1)
    ref = lbm.Solver(p)
    ref.step(700)
    a = lbm.Solver(p)
    a.step(300)
    snap = a.get_state(with_lo=True)
    a.close()
    b = lbm.Solver(p)
    b.set_state(*snap)
    b.step(400)
    for x, y in zip(ref.get_state(with_lo=True), b.get_state(with_lo=True)):
        assert np.array_equal(x, y)
    ref.close(); b.close()


def test_fields_on_device_equal_host_copies(lbm):
    import torch
    s = lbm.Solver(inputs.cavity(200, ny=130, precision=1))
    s.step(100)
    dev = s.fields(device=True)
    host = s.fields(device=False)
    for k in dev:
        assert np.array_equal(dev[k].cpu().numpy(), host[k])
    assert dev["T_f"].dtype == torch.float32
    part = s.fields(names=("f_l",), device=False)
    assert list(part) == ["f_l"] and np.array_equal(part["f_l"], host["f_l"])
    s.close()


def test_nonfinite_state_raises_sticky_unstable_flag(lbm):
    """A NaN planted in the state is caught by the kernel's check, reported as
    LBM_ERR_UNSTABLE, and later steps are refused; the context stays usable."""
    p = inputs.cavity(64, precision=1)
    s = lbm.Solver(p)
    f, g, h, dT = s.get_state()
    g[0, 10, 10] = np.nan
    s.set_state(f, g, h, dT)
    s.step(1)
    assert s.status() == -5
    with pytest.raises(lbm.LbmError) as e:
        s.step(1)
    assert e.value.code == -5
    s.close()
    ok = lbm.Solver(p)
    ok.step(10)
    assert ok.status() == 0
    ok.close()


def test_step_zero_and_negative(lbm):
    s = lbm.Solver(inputs.cavity(32, precision=1))
    s.step(0)
    assert s.steps == 0
    with pytest.raises(lbm.LbmError) as e:
        s.step(-1)
    assert e.value.code == -1
    s.close()


def test_lbm_create_with_cuda_allocator(lbm):
    """The stream-ordered CUDA allocator path (no PyTorch allocation hooks)."""
    p = inputs.cavity(64, precision=1)
    a = lbm.Solver(p, use_torch_alloc=False)
    b = lbm.Solver(p)
    a.step(50); b.step(50)
    for x, y in zip(a.get_state(with_lo=True), b.get_state(with_lo=True)):
        assert np.array_equal(x, y)
    a.close(); b.close()


VARIANTS = {"bgk": dict(thermal_collision=1), "bounce_back": dict(solid_scheme=1), "zeta_e": dict(zeta_e=0.6),
            "bounce_back_bgk": dict(solid_scheme=1, thermal_collision=1),
            "eq9": dict(ks_over_kl=0.5, cps_over_cpl=1.4),
            "eq9_bgk": dict(ks_over_kl=2.0, cps_over_cpl=0.8, thermal_collision=1),
            "eq9_zeta_e": dict(ks_over_kl=0.5, zeta_e=0.6),
            "ergun_F_phi": dict(F_phi=-1.0)}


@pytest.mark.parametrize("variant", sorted(VARIANTS))
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("qt", [5, 9])
def test_paper_variants_from_random_state(lbm, oracle_mod, variant, prec, qt):
    """The comparison variants of Sec. V (BGK thermal collision, bounce-back
    solid, explicit zeta_e) and the phase-dependent PCM properties of Eq. 9
    against the oracle, walled and periodic sides.
    Flow populations start near the rest equilibrium: without the blend the
    bounce-back scheme does not damp a state as far from equilibrium as
    f_i = 1/9 (the oracle and the kernel both reach |u| > 0.3 from it)."""
    for shape in ((131, 7, 0, 0), (64, 9, 1, 1)):
        nx, ny, px, py = shape
        p = inputs.cavity(max(nx, ny), ny=ny, precision=prec, thermal_q=qt, periodic_x=px, periodic_y=py,
                          L_char=100.0, Ra=1e7, **VARIANTS[variant])
        p["nx"] = nx
        s, o = _random_pair(lbm, oracle_mod, p, seed=nx + 3 * ny, f_base=W9[:, 0, 0])
        for n in (1, 2):
            s.step(n)
            o.run(n)
            _compare_states(s, o, prec, 1)
        fs, fo = s.fields(device=False), o.fields()
        for name, key in (("u_x", "u_x"), ("u_y", "u_y"), ("T_f", "T_f")):
            scale = max(np.abs(fo[key]).max(), 1e-3)
            assert np.abs(fs[name].astype(np.float64) - fo[key]).max() / scale < (1e-12 if prec == 0 else 5e-6)
        s.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
@pytest.mark.parametrize("qt", [5, 9])
def test_eq9_two_phase_melting_matches_oracle(lbm, oracle_mod, prec, tol, qt):
    """Melting into a subcooled solid with k_s = 2 k_l and c_ps = 1.5 c_pl
    (Eq. 9), exchange on: 6000 steps of the 200 x 4 conduction set-up."""
    p = inputs.conduction_1d(precision=prec, thermal_q=qt, T_init=-0.3, wall_T=[1.0, -0.3, 0.0, 0.0],
                             ks_over_kl=2.0, cps_over_cpl=1.5)
    s = lbm.Solver(p)
    o = oracle_mod.Oracle(p)
    s.step(6000)
    o.run(6000)
    fs, fo = s.fields(device=False), o.fields()
    for name in ("T_f", "T_s", "f_l"):
        key = "T_m" if name == "T_s" else name
        assert rel_l2(fs[name], fo[key]) < tol, name
    ds, do = s.diag(), o.diag()
    for k in ("melt_frac", "nu_hot", "enthalpy"):
        assert abs(ds[k] / do[k] - 1.0) < (1e-10 if prec == 0 else 1e-5), k
    assert 0.05 < do["melt_frac"] < 0.5
    s.close()


@pytest.mark.parametrize("prec,tol", [(1, 1e-5), (2, 3e-5), (3, 3e-5)])
def test_long_run_conservation_in_a_mushy_box(lbm, prec, tol):
    """20,000 steps of a random periodic box that settles on the melting
    plateau (the worst case for rounding: T_f pinned, a tiny persistent
    T_m - T_f), with the exchange on and off.  Total enthalpy drifts less than
    tol (measured: FP32 4.3e-6 and 2.5e-7, FP16 4.4e-7 and 1.3e-5, BF16 7.4e-6
    and 9.1e-6); with the exchange off the FP32 PCM enthalpy (float-float) is
    kept exactly."""
    for nu_i in (5.9, 0.0):
        p = inputs.periodic_box(256, 192, precision=prec, Ra=1e7, Nu_i=nu_i)
        F, G, Hm, dT = inputs.random_state(256, 192, 5, seed=9, H_range=(0.2, 1.4))
        s = lbm.Solver(p)
        s.set_state((F - W9).astype(np.float32), G.astype(np.float32), Hm.astype(np.float32), dT.astype(np.float32))
        d0 = s.diag()
        pcm0 = None
        if prec == 1:
            _, g, _, _, lo = s.get_state(with_lo=True)
            pcm0 = g.astype(np.float64).sum() + lo.astype(np.float64).sum()
        s.step(20_000)
        d1 = s.diag()
        assert s.status() == 0
        assert abs(d1["enthalpy"] / d0["enthalpy"] - 1) < tol
        if prec == 1 and nu_i == 0.0:
            _, g, _, _, lo = s.get_state(with_lo=True)
            assert abs((g.astype(np.float64).sum() + lo.astype(np.float64).sum()) / pcm0 - 1) < 1e-12
        s.close()


PAIR_SHAPES = [
    # node pairs forced: odd widths end in a single node, walls and periodic sides, blocks
    # with ragged tails, the smallest periodic pair (nx = 2), grids above 2^18 nodes
    (131, 7, 0, 0), (130, 9, 1, 1), (257, 4, 1, 0), (5, 3, 0, 1), (2, 2, 1, 1), (4, 5, 1, 0), (513, 520, 0, 0),
    (515, 511, 1, 1),
]


@pytest.mark.parametrize("shape", PAIR_SHAPES)
@pytest.mark.parametrize("variant", ["default", "eq9"])
def test_node_pair_kernel_from_random_state(lbm, oracle_mod, shape, variant):
    """The two-nodes-per-thread form of the fused step (LBM_STEP_FORM_PAIRS) in
    FP32 against the oracle, three steps from a random state; the Eq. 9
    variant compiles the per-node rates into it."""
    nx, ny, px, py = shape
    extra = VARIANTS["eq9"] if variant == "eq9" else {}
    p = inputs.cavity(max(nx, ny), ny=ny, precision=1, periodic_x=px, periodic_y=py, L_char=100.0, Ra=1e7,
                      **extra)
    p["nx"] = nx
    s, o = _random_pair(lbm, oracle_mod, p, seed=nx + 7 * ny)
    s.set_step_form(2)
    for n in (1, 2):
        s.step(n)
        o.run(n)
        _compare_states(s, o, 1, 1)
    s.close()


def test_step_forms_agree_over_a_graph_replayed_run(lbm):
    """Both step forms on the same cavity for 200 steps (graph replays and
    single launches): states within a few FP32 roundings of each other."""
    p = inputs.cavity(258, ny=130, precision=1)
    a, b = lbm.Solver(p).set_step_form(1), lbm.Solver(p).set_step_form(2)
    a.step(200)
    b.step(200)
    for x, y in zip(a.get_state(), b.get_state()):
        scale = max(np.abs(x).max(), 1e-3)
        assert np.abs(x.astype(np.float64) - y).max() / scale < 1e-5
    with pytest.raises(lbm.LbmError):
        a.set_step_form(4)
    a.close(); b.close()


TWO_STEP_SHAPES = [
    # (nx, ny, periodic_x, periodic_y): clamped last tiles, grids within one tile, the
    # smallest periodic grids, several tiles along both axes; blocks of 34 x H threads,
    # H from 4 to 13 and the 12-row build of grids with more than two tiles per SM
    # (520 x 300); H follows the grid and the SM count
    (31, 13, 0, 0), (61, 13, 1, 1), (30, 6, 0, 0), (3, 3, 0, 0), (1, 1, 1, 1), (2, 7, 1, 0),
    (97, 50, 0, 1), (131, 7, 1, 0), (257, 130, 0, 0), (300, 301, 1, 0), (256, 256, 0, 0), (520, 300, 1, 0),
]


@pytest.mark.parametrize("shape", TWO_STEP_SHAPES)
@pytest.mark.parametrize("qt", [5, 9])
@pytest.mark.parametrize("variant", ["default", "eq9", "bounce_back", "bgk", "zeta_e"])
def test_two_step_kernel_from_random_state(lbm, oracle_mod, shape, qt, variant):
    """Two time steps per launch (LBM_STEP_FORM_TWO_STEPS) in FP32: 4 and 8 steps
    (two and four launches) from a random state.  The states equal those of one
    step per launch bit for bit (the first step of each launch runs the same code
    on the same inputs, the second reads the same values from shared memory), and
    lie within FP32 rounding of the oracle: 4e-5 of array scale after 8 steps
    (measured 1.6e-5 on the 3 x 3 and 1 x 1 grids, about 1e-6 on the others; one
    step per launch has the same error)."""
    nx, ny, px, py = shape
    extra = VARIANTS[variant] if variant != "default" else {}
    p = inputs.cavity(max(nx, ny), ny=ny, precision=1, thermal_q=qt, periodic_x=px, periodic_y=py,
                      L_char=100.0, Ra=1e7, **extra)
    p["nx"] = nx
    assert lbm.step_form_for(p, 3) == 3
    s, o = _random_pair(lbm, oracle_mod, p, seed=nx + 5 * ny + qt, f_base=W9[:, 0, 0])
    ref = lbm.Solver(p).set_step_form(1)
    ref.load(s.save())
    s.set_step_form(3)
    # The bounce-back variant decides per node whether f_l <= 0.5.  Among the
    # 156,000 random mushy nodes of the 520 x 300 grid some lie within FP32
    # rounding of that threshold (3.6e-8 from it after 4 steps), where the FP32
    # kernel and the FP64 oracle can decide differently; there only the
    # bit-for-bit comparison with one step per launch applies.
    against_oracle = not (variant == "bounce_back" and nx * ny > 100_000)
    for n in (4, 4):
        s.step(n)
        ref.step(n)
        o.run(n)
        assert s.status() == 0
        for a, b in zip(s.get_state(), ref.get_state()):
            assert np.array_equal(a, b)
        if not against_oracle:
            continue
        f, g, h, dT = s.get_state()
        F, G, H, D = o.state()
        for a, b, name in ((f, F - W9, "f - w"), (g, G, "g"), (h, H, "h"), (dT, D, "dT")):
            scale = max(np.abs(b).max(), 1.0 if name == "dT" else 1e-3)
            assert np.abs(a.astype(np.float64) - b).max() / scale < 4e-5, (name, n)
    s.close()
    ref.close()


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("qt", [5, 9])
@pytest.mark.parametrize("variant", ["default", "eq9", "bounce_back", "bgk", "zeta_e"])
def test_two_step_kernel_16_bit_variants_equal_one_step(lbm, prec, qt, variant):
    """Two steps per launch in FP16/BF16 storage, every thermal lattice and
    variant, from a random state on walled and periodic sides: the states
    after 4 and 8 steps equal those of one step per launch bit for bit (the
    intermediate state sits in shared memory in the 16-bit encoding, as it
    would in a state copy)."""
    nx, ny = 97, 50
    extra = VARIANTS[variant] if variant != "default" else {}
    p = inputs.cavity(nx, ny=ny, precision=prec, thermal_q=qt, periodic_y=1, L_char=100.0, Ra=1e7, **extra)
    F, G, Hm, dT = inputs.random_state(nx, ny, qt, seed=300 + qt + prec, H_range=(0.0, 1.6), f_base=W9[:, 0, 0])
    s = lbm.Solver(p)
    s.set_state((F - W9).astype(np.float32), G.astype(np.float32), Hm.astype(np.float32), dT.astype(np.float32))
    ref = lbm.Solver(p).set_step_form(1)
    ref.load(s.save())
    s.set_step_form(3)
    for n in (4, 4):
        s.step(n)
        ref.step(n)
        assert s.status() == 0
        assert np.array_equal(s.save(), ref.save()), (n,)
    s.close()
    ref.close()


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_two_step_form_over_graph_replays_and_remainders(lbm, prec):
    """Two steps per launch against one step per launch on the same cavity:
    3 + 200 + 71 + 64 steps (single steps to state copy 0, graph replays, pairs of
    two-step launches, single remainders), states within a few roundings of the
    storage form; the exchange history is where checkpoints read it."""
    p = inputs.cavity(200, ny=70, precision=prec)
    a, b = lbm.Solver(p).set_step_form(1), lbm.Solver(p).set_step_form(3)
    rtol = {1: 1e-5, 2: 8 * 2.0 ** -11, 3: 8 * 2.0 ** -8}[prec]
    for n in (3, 200, 71, 64):
        a.step(n)
        b.step(n)
        assert b.status() == 0
        for x, y in zip(a.get_state(), b.get_state()):
            scale = max(np.abs(x).max(), 1e-3)
            assert np.abs(x.astype(np.float64) - y).max() / scale < rtol, n
    # a checkpoint of the two-step run resumes in a single-step run
    c = lbm.Solver(p).set_step_form(1)
    c.load(b.save())
    b.step(8)
    c.step(8)
    for x, y in zip(c.get_state(), b.get_state()):
        scale = max(np.abs(x).max(), 1e-3)
        assert np.abs(x.astype(np.float64) - y).max() / scale < rtol
    a.close(); b.close(); c.close()


def test_second_history_allocated_once_on_the_runs_allocator(lbm):
    """A run that steps two steps per launch takes one more allocation of
    lbm_history_bytes (plus the allocator's alignment slack) from its own
    allocator, at its first such lbm_step and only then; a run in one step per
    launch never does."""
    p = inputs.cavity(256, precision=1)
    assert lbm.step_form_for(p, 0) == 3
    s = lbm.Solver(p)
    live0 = dict(s._alloc.live)
    s.step(2)                                  # single steps only: nothing new
    assert s._alloc.live.keys() == live0.keys()
    s.step(64)
    new = [t for k, t in s._alloc.live.items() if k not in live0]
    assert len(new) == 1 and new[0].numel() - 256 == lbm.history_bytes(p)
    s.step(640)
    assert len(s._alloc.live) == len(live0) + 1
    q = dict(p, nx=512, ny=512)                # one step per launch at this size
    t = lbm.Solver(q)
    live1 = len(t._alloc.live)
    t.step(640)
    assert lbm.step_form_for(q, 0) == 1 and len(t._alloc.live) == live1
    s.close()
    t.close()
