"""Host-side checks of the C ABI (no GPU): the library builds, loads and exports
every entry point that include/lbm.h declares; its parameter map agrees with
the oracle's independent map; malformed and unstable inputs are rejected."""
import ctypes
import math
import re
from pathlib import Path

import pytest

from paper_1701_00702_gb300 import inputs

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lbm():
    from paper_1701_00702_gb300 import build, lbm as mod
    build.build()
    return mod


def declared_symbols():
    text = "\n".join(p.read_text() for p in (ROOT / "include").glob("*.h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)) - {"lbm_alloc_fn", "lbm_free_fn"})


def test_library_exports_every_declared_entry_point(lbm):
    L = lbm.lib()
    names = declared_symbols()
    assert "lbm_step" in names and "lbm_create" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


@pytest.mark.parametrize("make", [
    lambda: inputs.conduction_1d(),
    lambda: inputs.conduction_1d(thermal_q=9),
    lambda: inputs.cavity(256),
    lambda: inputs.cavity(1024, thermal_q=9),
    lambda: inputs.paper_cavity_defaults(),
    lambda: inputs.batch_draws(count=4)[3],
    lambda: dict(inputs.cavity(128), thermal_collision=1),
    lambda: dict(inputs.cavity(128, thermal_q=9), thermal_collision=1),
    lambda: dict(inputs.cavity(128, thermal_q=9), zeta_e=0.6),
    lambda: dict(inputs.cavity(128), zeta_e=1.8, solid_scheme=1),
    lambda: dict(inputs.cavity(128), ks_over_kl=0.5, cps_over_cpl=1.4, wall_T=[1.0, 0.1, 0.0, 0.0]),
    lambda: dict(inputs.cavity(128), F_phi=-1.0),
    lambda: inputs.conduction_1d(thermal_q=9, ks_over_kl=2.0, cps_over_cpl=1.5, T_init=-0.3,
                                 wall_T=[1.0, -0.3, 0.0, 0.0]),
])
def test_parameter_map_matches_oracle(lbm, oracle_mod, make):
    p = make()
    d = lbm.derive(p)
    lc = oracle_mod.lattice_config(p)
    keys = ["k_m", "rho_m", "L_a", "h_v", "alpha_fref", "alpha_mref", "c_fref", "c_mref", "d_p"]
    if p["flow"]:
        keys += ["nu_f", "nu_e", "gbeta", "K", "F_phi"]
    for k in keys:
        assert math.isclose(d[k], lc[k], rel_tol=1e-15, abs_tol=0.0), k
    q = lc["qt"]
    assert d["zeta"][:q] == pytest.approx(lc["zeta"][:q], rel=1e-15)
    assert d["eta"][:q] == pytest.approx(lc["eta"][:q], rel=1e-15)
    if p["flow"]:
        assert d["s"] == pytest.approx(lc["s"], rel=1e-15)
    for side in range(4):
        assert d["H_wall"][side] == pytest.approx(oracle_mod.H_of_T(p, p["wall_T"][side]), rel=1e-15, abs=1e-15)
    assert math.isclose(d["k_s"], lc["k_s"], rel_tol=1e-15) and math.isclose(d["c_ps"], lc["c_ps"], rel_tol=1e-15)
    assert math.isclose(d["H_fs"], lc["c_ps"] * lc["T_fs"], rel_tol=1e-15, abs_tol=1e-300)
    za_s = 1.0 / (0.5 + lc["k_s"] / (lc["rho_l"] * lc["c_fref"]) / lc["csT2"])      # Eq. A19 with k_s
    assert math.isclose(d["zeta_a_solid"], za_s, rel_tol=1e-15)


@pytest.mark.parametrize("change", [
    dict(nx=0), dict(ny=-1), dict(nx=2), dict(thermal_q=7), dict(precision=5), dict(porosity=1.0),
    dict(porosity=0.0), dict(Ste=0.0), dict(k_f=-1.0), dict(T_solidus=0.4, T_liquidus=0.3),
    dict(T_hot=0.0, T_cold=0.0), dict(T_hot=0.0, T_cold=1.0), dict(varpi=1.0), dict(Da=0.0),
    dict(Pr=float("nan")), dict(wall_kind=[0, 0, 2, 1]), dict(nx=65537), dict(nx=40000, ny=40000),
    dict(thermal_collision=2), dict(solid_scheme=-1), dict(zeta_e=-0.5), dict(ks_over_kl=0.0),
    dict(cps_over_cpl=-1.0), dict(ks_over_kl=float("inf")),
])
def test_malformed_parameters_are_rejected(lbm, change):
    p = inputs.cavity(64)
    p.update(change)
    with pytest.raises(lbm.LbmError) as e:
        lbm.derive(p)
    assert e.value.code == -1
    assert lbm.state_bytes(p) == -1


@pytest.mark.parametrize("change", [
    dict(k_f=0.2),                                # large diffusivity: exchange rate h_v grows past 1
    dict(cfref_over_cpl=1.6, thermal_q=5),        # varpi c_f,ref >= c_pl (D2Q5 analogue of Remark I)
    dict(cfref_over_cpl=1.85, thermal_q=9),       # Remark I
    dict(Nu_i=500.0),                             # explicit exchange rate >= 1
    dict(zeta_e=2.0),                             # an explicit zeta_e outside (0, 2)
])
def test_unstable_parameters_are_rejected(lbm, change):
    p = inputs.cavity(64)
    p.update(change)
    with pytest.raises(lbm.LbmError) as e:
        lbm.derive(p)
    assert e.value.code == -2


def test_size_limits(lbm):
    p = inputs.periodic_box(32768, 32768)
    assert lbm.state_bytes(p) > 0
    p = inputs.periodic_box(32768, 32769)
    assert lbm.state_bytes(p) == -1
    p = inputs.periodic_box(1, 1, L_char=100.0)
    assert lbm.state_bytes(p) > 0


def test_history_bytes_cover_one_array_of_the_row_pitch(lbm):
    """lbm_history_bytes: one exchange-history array, rows padded to the
    128-node chunk pitch, 4 bytes per node (8 in FP64), 256-byte aligned."""
    assert lbm.history_bytes(inputs.cavity(256, precision=1)) == 256 * 256 * 4
    assert lbm.history_bytes(inputs.cavity(200, ny=70, precision=2)) == 256 * 70 * 4
    assert lbm.history_bytes(inputs.cavity(129, ny=3, precision=0)) == 256 * 3 * 8
    assert lbm.history_bytes(dict(inputs.cavity(64), nx=0)) == -1


def test_state_bytes_account_for_both_copies(lbm):
    p = inputs.cavity(2048)
    b = lbm.state_bytes(p)
    per_node = (2 * (9 + 5 + 5 + 1) + 1) * 4     # two copies of 19 populations + the low part of g_0, history
    assert per_node * 2048 * 2048 <= b < per_node * 2048 * 2048 * 1.01


def test_strerror_names_every_code(lbm):
    for code in range(0, -8, -1):
        s = lbm.lib().lbm_strerror(code).decode()
        assert s and s != "unknown status code"
    assert lbm.lib().lbm_strerror(-99).decode() == "unknown status code"


def test_create_without_gpu_fails_cleanly(lbm):
    """On a host without a GPU lbm_create reports an error instead of crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lbm.lib().lbm_create(ctypes.byref(lbm.to_struct(inputs.cavity(16))), None, ctypes.byref(h))
    assert rc in (-3, -4) and not h.value


@pytest.mark.parametrize("params,form,expected", [
    # automatic: node pairs for FP16/BF16 runs of the default configuration from 1536 x 1024 nodes
    (dict(n=2048, precision=2), 0, 2),
    (dict(n=2048, precision=3), 0, 2),
    (dict(n=2048, ny=4096, precision=2), 0, 2),
    (dict(n=2048, ny=1024, precision=2), 0, 2),
    (dict(n=1536, ny=1024, precision=3), 0, 2),
    (dict(n=1536, ny=1023, precision=2), 0, 1),            # one row short of 1,572,864 nodes
    (dict(n=1024, precision=2), 0, 1),
    (dict(n=2048, precision=0), 0, 1),
    (dict(n=2048, precision=2, thermal_q=9), 0, 1),
    (dict(n=2048, precision=2, flow=0), 0, 1),
    (dict(n=2048, precision=2, solid_scheme=1), 0, 1),     # bounce-back variant
    (dict(n=2048, precision=2, ks_over_kl=0.5), 0, 2),      # Eq. 9 rates: compiled into both forms
    # forced
    (dict(n=64, precision=1), 2, 2),
    (dict(n=3, precision=3, L_char=100.0), 2, 2),
    (dict(n=64, precision=0), 2, 1),                        # no FP64 node-pair kernel
    (dict(n=64, precision=1, thermal_q=9), 2, 1),
    (dict(n=2048, precision=2), 1, 1),
    # automatic two steps per launch (D2Q5, flow, FP32/FP16/BF16): up to 320 x 320 nodes, and
    # FP32 from 786,432 nodes (state beyond L2); between them one step per launch
    (dict(n=256, precision=1), 0, 3),
    (dict(n=320, precision=2), 0, 3),
    (dict(n=64, precision=3), 0, 3),
    (dict(n=320, ny=321, precision=1), 0, 1),
    (dict(n=352, precision=2), 0, 1),
    (dict(n=512, precision=1), 0, 1),
    (dict(n=768, precision=1), 0, 1),
    (dict(n=1024, ny=767, precision=1), 0, 1),
    (dict(n=1024, ny=768, precision=1), 0, 3),
    (dict(n=1024, precision=1), 0, 3),
    (dict(n=2048, precision=1), 0, 3),
    (dict(n=4096, ny=256, precision=1, solid_scheme=1), 0, 3),
    (dict(n=1024, precision=2), 0, 1),                     # 16-bit: one node per thread, then pairs
    (dict(n=256, precision=0), 0, 1),
    (dict(n=256, precision=1, thermal_q=9), 0, 1),
    (dict(n=256, precision=1, flow=0), 0, 1),
    (dict(n=256, precision=1), 1, 1),
    (dict(n=256, precision=1), 2, 2),
    # forced two steps per launch: runs with flow in FP32/FP16/BF16 storage, any lattice and variant
    (dict(n=256, precision=1), 3, 3),
    (dict(n=256, precision=2, thermal_q=9), 3, 3),
    (dict(n=3, precision=3, L_char=100.0), 3, 3),
    (dict(n=2048, precision=2, solid_scheme=1), 3, 3),
    (dict(n=256, precision=0), 3, 1),                       # no FP64 two-step kernel
    (dict(n=256, precision=1, flow=0), 3, 1),
])
def test_step_form_rule(lbm, params, form, expected):
    """lbm_step_form_for reports the kernel form lbm_step takes (the same rule
    the launcher uses), with no GPU."""
    params = dict(params)
    n = params.pop("n")
    p = inputs.cavity(n, **params)
    assert lbm.step_form_for(p, form) == expected


def test_step_form_query_rejects_bad_input(lbm):
    with pytest.raises(lbm.LbmError):
        lbm.step_form_for(inputs.cavity(64), 4)
    with pytest.raises(lbm.LbmError):
        lbm.step_form_for(dict(inputs.cavity(64), nx=0), 0)


@pytest.mark.parametrize("prec,flow,ok", [(1, 1, True), (2, 1, True), (3, 1, True), (0, 1, False), (1, 0, False)])
def test_server_takes_map_5_only_for_runs_with_flow_in_32_or_16_bit_storage(lbm, prec, flow, ok):
    """Host-only: lbm_server_configure accepts map 5 (grouped two-step
    launches) for servers of runs with flow in FP32/FP16/BF16 storage and
    refuses it otherwise; maps 0-4 are always accepted."""
    L = lbm.lib()
    s = ctypes.c_void_p()
    no_alloc, no_free = lbm.ALLOC_FN(), lbm.FREE_FN()        # NULL hooks: the CUDA stream-ordered allocator
    assert L.lbm_server_create(1 << 30, 4, 1, 64, prec, 5, flow, None, no_alloc, no_free, None, ctypes.byref(s)) == 0
    assert (L.lbm_server_configure(s, 128, 5) == 0) == ok
    assert L.lbm_server_configure(s, 128, 4) == 0
    assert L.lbm_server_configure(s, 128, 6) != 0
    L.lbm_server_destroy(s)


def test_server_budget_counts_the_second_history_under_map_5(lbm):
    """Host-only: a request whose state alone fills the budget is taken under
    map 4 and refused under map 5, which also holds its second history array
    (lbm_history_bytes)."""
    L = lbm.lib()
    p = inputs.cavity(128, precision=2)
    budget = lbm.state_bytes(p)
    struct = lbm.to_struct(p)
    for mapping, accepted in ((4, True), (5, False)):
        s = ctypes.c_void_p()
        assert L.lbm_server_create(budget, 4, 1, 64, 2, 5, 1, None, lbm.ALLOC_FN(), lbm.FREE_FN(), None,
                                   ctypes.byref(s)) == 0
        assert L.lbm_server_configure(s, 128, mapping) == 0
        rid = ctypes.c_int64()
        assert (L.lbm_server_submit(s, ctypes.byref(struct), 100, ctypes.byref(rid)) == 0) == accepted
        L.lbm_server_destroy(s)
