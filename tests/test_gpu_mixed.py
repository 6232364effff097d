"""16-bit storage forms (FP16 and BF16 populations, FP32 rest populations and
arithmetic) against the FP64 oracle.

Tolerances: one step from a state already on the 16-bit grid agrees to the
storage rounding of its outputs (2^-11 relative for FP16, 2^-8 for BF16, of
each array's scale, with a factor 2 margin); long runs are assessed on the
integral quantities the method's stated target names: melt fraction and
hot-wall Nusselt number within 1e-3 relative of the FP64 oracle for FP16.
BF16 keeps 8 significant bits and is held to 1e-2 (measured: 1.4e-3 on the
cavity melt fraction, 5.2e-3 on the conduction-case Nusselt number).
"""
import numpy as np
import pytest

from paper_1701_00702_gb300 import inputs

pytestmark = pytest.mark.gpu

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]   # Eq. 27 weights
F16, BF16 = 2, 3


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1701_00702_gb300 import build, lbm as mod
    build.build()
    return mod


def to_bf16_grid(a):
    """Round float32 values to the nearest bfloat16 (ties to even), as float32."""
    b = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def on_grid(a, prec, scale=1.0):
    a = np.asarray(a, np.float32)
    if prec == F16:
        return (np.asarray(a * scale, np.float16).astype(np.float32) / scale).astype(np.float32)
    return to_bf16_grid(a)


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.sqrt(((a - b) ** 2).sum() / max((b * b).sum(), 1e-300)))


@pytest.mark.parametrize("prec,rtol", [(F16, 2 * 2.0 ** -11), (BF16, 2 * 2.0 ** -8)])
@pytest.mark.parametrize("qt", [5, 9])
@pytest.mark.parametrize("shape", [(131, 7, 0, 0), (130, 9, 1, 1), (3, 3, 0, 0), (257, 4, 0, 1)])
def test_one_step_from_random_state(lbm, oracle_mod, prec, rtol, qt, shape):
    nx, ny, px, py = shape
    p = inputs.cavity(max(nx, ny), ny=ny, precision=prec, thermal_q=qt, periodic_x=px, periodic_y=py,
                      L_char=100.0, Ra=1e7)
    p["nx"] = nx
    lc = oracle_mod.lattice_config(p)
    F, G, Hm, dT = inputs.random_state(nx, ny, qt, seed=nx + 7 * ny,
                                       H_range=(lc["T_fs"] - 0.3, lc["T_fl"] + lc["L_a"] + 0.3))
    Fd = on_grid(F - W9, prec, 1024.0)
    G = G.astype(np.float32)
    Hm = Hm.astype(np.float32)
    G[1:] = on_grid(G[1:], prec)
    Hm[1:] = on_grid(Hm[1:], prec)
    dT = dT.astype(np.float32)
    s = lbm.Solver(p)
    s.set_state(Fd, G, Hm, dT)
    f0, g0, h0, d0 = s.get_state()
    assert np.array_equal(f0, Fd)                        # flow: exact round trip
    for a, b in ((g0, G), (h0, Hm)):                     # thermal movers: one 16-bit rounding of the deviation
        assert np.array_equal(a[0], b[0])
        assert np.abs(a[1:] - b[1:]).max() <= 2 * rtol * np.abs(b[1:]).max()
    G, Hm = g0.copy(), h0.copy()                         # the oracle starts from what the solver holds
    o = oracle_mod.Oracle(p)
    o.set_state(Fd.astype(np.float64) + W9, G.astype(np.float64), Hm.astype(np.float64), dT.astype(np.float64))
    s.step(1)
    o.run(1)
    f1, g1, h1, d1 = s.get_state()
    Fo, Go, Ho, Do = o.state()
    for a, b, name in ((f1, Fo - W9, "f - w"), (g1, Go, "g"), (h1, Ho, "h")):
        err = np.abs(a.astype(np.float64) - b).max() / max(np.abs(b).max(), 1e-3)
        assert err < rtol * 4, (name, err)
    assert np.abs(d1 - Do).max() < 1e-5
    s.close()


@pytest.mark.parametrize("prec", [F16, BF16, 1, 0])
def test_checkpoint_resume_is_bitwise(lbm, prec):
    p = inputs.cavity(96, ny=64, precision=prec)
    a = lbm.Solver(p)
    a.step(200)
    snap = a.save()
    ref = lbm.Solver(p)
    ref.step(500)
    b = lbm.Solver(p)
    b.load(snap)
    assert b.steps == 200
    b.step(300)
    assert np.array_equal(ref.save(), b.save())
    other = lbm.Solver(inputs.cavity(96, ny=65, precision=prec))
    with pytest.raises(lbm.LbmError):
        other.load(snap)
    a.close(); b.close(); ref.close(); other.close()


@pytest.mark.parametrize("prec", [F16, BF16])
def test_periodic_box_conservation(lbm, prec):
    p = inputs.periodic_box(256, 192, precision=prec, Ra=1e7)
    F, G, Hm, dT = inputs.random_state(256, 192, 5, seed=9, H_range=(0.2, 1.4))
    s = lbm.Solver(p)
    s.set_state((F - W9).astype(np.float32), G.astype(np.float32), Hm.astype(np.float32), dT.astype(np.float32))
    d0 = s.diag()
    s.step(500)
    d1 = s.diag()
    # the stored rest population closes the balance with the movers as readers
    # decode them, so enthalpy is kept to FP32 rounding (measured 3e-8 / 1.4e-8)
    assert abs(d1["enthalpy"] / d0["enthalpy"] - 1) < 1e-6
    assert abs(d1["mass"] / d0["mass"] - 1) < 1e-3
    s.close()


TOL = {F16: 1e-3, BF16: 1e-2}


@pytest.mark.parametrize("prec", [F16, BF16])
def test_cavity_melt_fraction_and_nusselt_vs_fp64_oracle(lbm, oracle_mod, prec):
    """256 x 256 square-cavity melting with natural convection, 4,000 steps:
    melt fraction and hot-wall Nusselt number of the 16-bit form within 1e-3
    relative of the FP64 oracle."""
    p64 = inputs.cavity(256, precision=0)
    p = inputs.cavity(256, precision=prec)
    s = lbm.Solver(p)
    s.step(4000)
    assert s.status() == 0
    d = s.diag()
    o = oracle_mod.Oracle(p64).run(4000)
    do = o.diag()
    assert abs(d["melt_frac"] / do["melt_frac"] - 1) < TOL[prec]
    assert abs(d["nu_hot"] / do["nu_hot"] - 1) < TOL[prec]
    f, fo = s.fields(device=False), o.fields()
    assert rel_l2(f["T_f"], fo["T_f"]) < 1e-2
    s.close()


@pytest.mark.parametrize("prec", [F16, BF16])
def test_conduction_melting_vs_fp64_oracle(lbm, oracle_mod, prec):
    p = inputs.conduction_1d(precision=prec)
    s = lbm.Solver(p)
    s.step(20000)
    o = oracle_mod.Oracle(inputs.conduction_1d(precision=0)).run(20000)
    d, do = s.diag(), o.diag()
    assert abs(d["melt_frac"] / do["melt_frac"] - 1) < TOL[prec]
    assert abs(d["nu_hot"] / do["nu_hot"] - 1) < TOL[prec]
    s.close()


@pytest.mark.parametrize("prec,rtol", [(F16, 2 * 2.0 ** -11), (BF16, 2 * 2.0 ** -8)])
def test_full_size_sampled_parity_2048(lbm, oracle_mod, prec, rtol):
    """The 16-bit forms on the 2048 x 2048 cavity in the benchmark's launch
    configuration: one step from a random state (as the solver holds it after
    encoding) against the oracle at sampled nodes, all edges and corners plus
    random interior nodes."""
    n = 2048
    p = inputs.cavity(n, precision=prec)
    lc = oracle_mod.lattice_config(p)
    F, G, Hm, dT = inputs.random_state(n, n, 5, seed=2049, H_range=(lc["T_fs"] - 0.3, lc["T_fl"] + lc["L_a"] + 0.3))
    s = lbm.Solver(p)
    s.set_state(on_grid(F - W9, prec, 1024.0), G.astype(np.float32), Hm.astype(np.float32), dT.astype(np.float32))
    del F, G, Hm
    f0, g0, h0, d0 = s.get_state()                        # the oracle starts from what the solver holds
    s.step(1)
    f1, g1, h1, d1 = s.get_state()
    o = oracle_mod.Oracle(p)
    o.set_state(f0.astype(np.float64) + W9, g0.astype(np.float64), h0.astype(np.float64), d0.astype(np.float64))
    rng = np.random.default_rng(11)
    edge = np.arange(n)
    xs = np.concatenate([edge, edge, np.zeros(n, int), np.full(n, n - 1), rng.integers(0, n, 20000)])
    ys = np.concatenate([np.zeros(n, int), np.full(n, n - 1), edge, edge, rng.integers(0, n, 20000)])
    fo, go, ho, do = o.step_nodes(xs, ys)
    fo = fo - W9[:, 0, 0][None, :]
    for a, b, name in ((f1[:, ys, xs].T, fo, "f - w"), (g1[:, ys, xs].T, go, "g"), (h1[:, ys, xs].T, ho, "h")):
        err = np.abs(a.astype(np.float64) - b).max() / max(np.abs(b).max(), 1e-3)
        assert err < rtol * 4, (name, err)
    assert np.abs(d1[ys, xs] - do).max() < 1e-5
    s.close()


@pytest.mark.parametrize("prec", [F16, BF16])
def test_config2_size_against_fp32(lbm, prec):
    """The 1024 x 1024 cavity (the mixed-precision workload's size), 4,000 steps:
    melt fraction and hot-wall Nusselt number of the 16-bit form within the
    mixed-form tolerance of the FP32 path on the same GPU (which the parity
    tests hold to 1e-5 of the FP64 oracle)."""
    d = {}
    for q in (1, prec):
        s = lbm.Solver(inputs.cavity(1024, precision=q))
        s.step(4000)
        assert s.status() == 0
        d[q] = s.diag()
        s.close()
    assert abs(d[prec]["melt_frac"] / d[1]["melt_frac"] - 1) < TOL[prec]
    assert abs(d[prec]["nu_hot"] / d[1]["nu_hot"] - 1) < TOL[prec]


@pytest.mark.parametrize("prec,rtol", [(F16, 2 * 2.0 ** -11), (BF16, 2 * 2.0 ** -8)])
@pytest.mark.parametrize("shape", [(131, 7, 0, 0), (130, 9, 1, 1), (5, 3, 0, 1), (513, 520, 0, 0)])
@pytest.mark.parametrize("eq9", [0, 1])
def test_node_pair_kernel_one_step(lbm, oracle_mod, prec, rtol, shape, eq9):
    """The two-nodes-per-thread form (LBM_STEP_FORM_PAIRS, automatic for the
    16-bit forms from 1536 x 1024 nodes) in FP16 and BF16: one step from a random
    state against the oracle, with and without the Eq. 9 per-node rates."""
    nx, ny, px, py = shape
    extra = dict(ks_over_kl=0.5, cps_over_cpl=1.4) if eq9 else {}
    p = inputs.cavity(max(nx, ny), ny=ny, precision=prec, periodic_x=px, periodic_y=py, L_char=100.0, Ra=1e7,
                      **extra)
    p["nx"] = nx
    lc = oracle_mod.lattice_config(p)
    F, G, Hm, dT = inputs.random_state(nx, ny, 5, seed=nx + ny, H_range=(lc["T_fs"] - 0.3, lc["T_fl"] + lc["L_a"] + 0.3))
    s = lbm.Solver(p).set_step_form(2)
    s.set_state(on_grid(F - W9, prec, 1024.0), G.astype(np.float32), Hm.astype(np.float32), dT.astype(np.float32))
    f0, g0, h0, d0 = s.get_state()
    o = oracle_mod.Oracle(p)
    o.set_state(f0.astype(np.float64) + W9, g0.astype(np.float64), h0.astype(np.float64), d0.astype(np.float64))
    s.step(1)
    o.run(1)
    f1, g1, h1, d1 = s.get_state()
    Fo, Go, Ho, Do = o.state()
    for a, b, name in ((f1, Fo - W9, "f - w"), (g1, Go, "g"), (h1, Ho, "h")):
        err = np.abs(a.astype(np.float64) - b).max() / max(np.abs(b).max(), 1e-3)
        assert err < rtol * 4, (name, err)
    assert np.abs(d1 - Do).max() < 1e-5
    s.close()
