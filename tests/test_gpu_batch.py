"""Batched stepping of unequal cavities.

Map 3 launches lbm_step's own kernel per run, so a batched step equals
lbm_step bit for bit in every storage mode; so does map 5, whose grouped
two-step launches run the two-step kernel's code (equal to one step per
launch bit for bit) and whose single steps take each run's one-step kernel.
Maps 0-2 inline the same per-node code into the tile kernel and map 4 into
the grouped kernel (runs below 2^20 nodes), where the compiler may fuse a few
multiply-adds differently: their states agree with lbm_step to within a few
roundings of the storage format (TILE_TOL, relative to each array's scale).
"""

EXACT_MAPS = (3, 5)
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


def _mixed_params(prec, qt=5):
    draws = inputs.batch_draws(count=5, seed=7, n_lo=40, n_hi=200)
    shapes = [(64, 64), (96, 80), (130, 70), (257, 33), (200, 200)]
    out = []
    for p, (nx, ny) in zip(draws, shapes):
        p.update(nx=nx, ny=ny, precision=prec, thermal_q=qt, L_char=float(nx))
        out.append(p)
    out[3].update(periodic_y=1)                # walls only in x for one run
    return out


@pytest.mark.parametrize("prec,qt", [(1, 5), (2, 5), (0, 9), (3, 5)])
def test_batch_equals_individual_runs(lbm, prec, qt):
    ps = _mixed_params(prec, qt)
    batch_runs = [lbm.Solver(p) for p in ps]
    solo = [lbm.Solver(p) for p in ps]
    b = lbm.Batch(batch_runs, autotune=True)
    info = b.info()
    assert info["n_tiles"] > 0 and info["tuned_us_per_step"] > 0
    b.step(3)
    b.step(150)                 # odd start: single launches, then captured graphs
    for s in solo:
        s.step(153)
    exact = info["mapping"] in ("single-run kernel chains", "grouped launches, two steps each")
    for x, y in zip(batch_runs, solo):
        assert x.steps == y.steps == 153
        assert _same_state(x, y, exact, prec)
    b.close()
    for s in batch_runs + solo:
        s.close()


TILE_TOL = {0: 1e-12, 1: 2e-6, 2: 1e-3, 3: 8e-3}   # FP64, FP32, FP16, BF16


def _same_state(a, b, exact, prec=1):
    """Equal checkpoints (exact), or states within TILE_TOL[prec] of each
    array's scale (tile maps)."""
    if exact:
        return np.array_equal(a.save(), b.save())
    fa, ga, ha, da, la = a.get_state(with_lo=True)
    fb, gb, hb, db, lb = b.get_state(with_lo=True)
    ga, gb = ga.astype(np.float64), gb.astype(np.float64)
    if la is not None:      # the rest population is the float-float pair g_0 + lo: compare the sum
        ga[0] += la
        gb[0] += lb
    for x, y in ((fa, fb), (ga, gb), (ha, hb), (da, db)):
        if x is None:
            continue
        scale = max(float(np.abs(y).max()), 1e-3)
        if np.abs(x.astype(np.float64) - y).max() > TILE_TOL[prec] * scale:
            return False
    return True


@pytest.mark.parametrize("prec", [1, 2])
def test_every_map_gives_the_same_state(lbm, prec):
    ps = _mixed_params(prec)
    ref = [lbm.Solver(p) for p in ps]
    for s in ref:
        s.step(40)
    for cap in (32, 64, 128, 256):
        for mapping in (0, 1, 2, 3, 4, 5):
            runs = [lbm.Solver(p) for p in ps]
            b = lbm.Batch(runs, autotune=False).configure(cap, mapping)
            b.step(40)
            for r, w in zip(runs, ref):
                assert _same_state(r, w, mapping in EXACT_MAPS, prec), (cap, mapping)
            b.close()
            for r in runs:
                r.close()


def test_batch_rejects_mixed_runs(lbm):
    a = lbm.Solver(inputs.cavity(64, precision=1))
    c = lbm.Solver(inputs.cavity(64, precision=2))
    with pytest.raises(lbm.LbmError) as e:
        lbm.Batch([a, c])
    assert e.value.code == -1
    with pytest.raises(lbm.LbmError):
        lbm.Batch([a, a])
    for s in (a, c):
        s.close()


def test_runs_at_different_step_parities_batch_correctly(lbm):
    """Runs that joined at different times (odd and even step counts) advance
    together and match their individually stepped twins."""
    ps = _mixed_params(1)
    runs = [lbm.Solver(p) for p in ps]
    twins = [lbm.Solver(p) for p in ps]
    for k, (r, t) in enumerate(zip(runs, twins)):
        r.step(k)
        t.step(k)
    b = lbm.Batch(runs, autotune=False)
    b.step(1)
    b.step(130)
    for t in twins:
        t.step(131)
    for r, t in zip(runs, twins):
        assert r.steps == t.steps
        assert _same_state(r, t, exact=False)   # FP32, default map 0
    b.close()
    for s in runs + twins:
        s.close()


def test_batch_of_64_cavities_advances_and_stays_finite(lbm):
    """The 64-cavity workload (sides 64..512, mixed porosity, Da, Ra, Ste) in FP16."""
    runs = [lbm.Solver(dict(p, precision=2)) for p in inputs.batch_draws(count=64)]
    b = lbm.Batch(runs, autotune=True)
    b.step(500)
    for r in runs:
        assert r.status() == 0 and r.steps == 500
        d = r.diag()
        assert np.isfinite(d["nu_hot"]) and 0.0 <= d["melt_frac"] <= 1.0
    b.close()
    for r in runs:
        r.close()


W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]   # Eq. 27 weights


@pytest.mark.parametrize("prec,qt", [(1, 5), (1, 9), (2, 5), (2, 9), (0, 9)])
@pytest.mark.parametrize("mapping", [0, 1, 2, 3, 4, 5])
def test_batch_from_random_states(lbm, prec, qt, mapping):
    """Runs holding random states (populations spread over solid, mushy and
    liquid nodes, flow near rest) advance in a batch exactly as alone (21
    steps: under map 5 five pairs of two-step launches and one single step;
    FP64 batches have no map 5)."""
    shapes = [(131, 7, 0, 0), (70, 33, 1, 0), (64, 64, 1, 1)]
    ps = [inputs.cavity(nx, ny=ny, precision=prec, thermal_q=qt, periodic_x=px, periodic_y=py, L_char=100.0,
                        Ra=1e7) for nx, ny, px, py in shapes]
    runs, solo = [], []
    for k, p in enumerate(ps):
        F, G, Hm, dT = inputs.random_state(p["nx"], p["ny"], qt, seed=40 + k, H_range=(-0.2, 1.6),
                                           f_base=W9.ravel())
        for dst in (runs, solo):
            s = lbm.Solver(p)
            s.set_state(F - W9, G, Hm, dT)
            dst.append(s)
    if mapping == 5 and prec == 0:
        b = lbm.Batch(runs, autotune=False)
        with pytest.raises(lbm.LbmError):
            b.configure(128, 5)
        b.close()
        for s in runs + solo:
            s.close()
        return
    b = lbm.Batch(runs, autotune=False).configure(128, mapping)
    b.step(21)
    for s in solo:
        s.step(21)
    for r, s in zip(runs, solo):
        assert _same_state(r, s, mapping in EXACT_MAPS, prec)
    b.close()
    for s in runs + solo:
        s.close()


def test_block_shapes_under_map_3_change_no_result(lbm):
    """Per-run block shapes under map 3 (the tuner's per-size-class choice)
    leave every run bit for bit equal to lbm_step."""
    shapes = [(131, 7, 0, 0), (70, 33, 1, 0), (64, 64, 1, 1), (300, 45, 0, 0)]
    ps = [inputs.cavity(nx, ny=ny, precision=1, periodic_x=px, periodic_y=py, L_char=100.0, Ra=1e7)
          for nx, ny, px, py in shapes]
    runs, solo = [], []
    for k, p in enumerate(ps):
        F, G, Hm, dT = inputs.random_state(p["nx"], p["ny"], 5, seed=60 + k, H_range=(-0.2, 1.6), f_base=W9.ravel())
        for dst in (runs, solo):
            s = lbm.Solver(p)
            s.set_state(F - W9, G, Hm, dT)
            dst.append(s)
    b = lbm.Batch(runs, autotune=False).configure(128, 3)
    for r, blk in enumerate([(64, 4), (32, 2), (256, 1), (64, 1)]):
        b.set_block(r, *blk)
    assert b.blocks() == [(64, 4), (32, 2), (256, 1), (64, 1)]
    with pytest.raises(lbm.LbmError):
        b.set_block(0, 16, 16)
    b.step(70)
    for s in solo:
        s.step(70)
    for r, s in zip(runs, solo):
        assert np.array_equal(r.save(), s.save())
    b.close()
    tuned = lbm.Batch(runs, autotune=True)
    assert all(blk in [(128, 2), (64, 4), (32, 8), (256, 1), (128, 1), (64, 2), (32, 4), (64, 1), (32, 2)]
               for blk in tuned.blocks())
    tuned.close()
    for s in runs + solo:
        s.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_node_pair_runs_under_map_3_equal_lbm_step(lbm, prec):
    """Runs set to the node-pair step form keep it inside a map-3 batch, bit for
    bit equal to lbm_step; runs left on one node per thread beside them too."""
    shapes = [(131, 7, 0, 0), (70, 33, 1, 0), (64, 64, 1, 1)]
    ps = [inputs.cavity(nx, ny=ny, precision=prec, periodic_x=px, periodic_y=py, L_char=100.0, Ra=1e7)
          for nx, ny, px, py in shapes]
    runs, solo = [], []
    for k, p in enumerate(ps):
        F, G, Hm, dT = inputs.random_state(p["nx"], p["ny"], 5, seed=80 + k, H_range=(-0.2, 1.6), f_base=W9.ravel())
        for dst in (runs, solo):
            s = lbm.Solver(p).set_step_form(2 if k != 1 else 1)
            s.set_state(F - W9, G, Hm, dT)
            dst.append(s)
    b = lbm.Batch(runs, autotune=False).configure(128, 3)
    b.step(70)
    for s in solo:
        s.step(70)
    for r, s in zip(runs, solo):
        assert _same_state(r, s, True, prec)
    b.close()
    for s in runs + solo:
        s.close()


@pytest.mark.parametrize("mapping", [0, 3, 4, 5])
def test_a_run_stepped_on_its_own_between_batch_steps(lbm, mapping):
    """lbm_step on a member run between batched steps (same stream) moves that
    run to the other state copy; the next batched step follows it instead of
    advancing the stale copy, and every run matches its individually stepped
    twin."""
    ps = _mixed_params(1)
    runs = [lbm.Solver(p) for p in ps]
    twins = [lbm.Solver(p) for p in ps]
    b = lbm.Batch(runs, autotune=False).configure(128, mapping)
    b.step(70)                  # one replayed graph and six single steps
    runs[1].step(1)             # an odd number of the run's own steps
    runs[3].step(2)
    b.step(70)
    for k, t in enumerate(twins):
        t.step(140 + (1 if k == 1 else 2 if k == 3 else 0))
    for r, t in zip(runs, twins):
        assert r.steps == t.steps
        assert _same_state(r, t, mapping in EXACT_MAPS)
    b.close()
    for s in runs + twins:
        s.close()


# one step from a state on the storage grid, as the single-run parity tests:
# FP64 1e-12, FP32 5e-6, FP16/BF16 four 16-bit roundings (2 x 2^-11, 2 x 2^-8)
ORACLE_TOL = {0: 1e-12, 1: 5e-6, 2: 8 * 2.0 ** -11, 3: 8 * 2.0 ** -8}


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("mapping", [0, 1, 2, 4])
def test_tile_maps_match_the_oracle(lbm, oracle_mod, prec, mapping):
    """The tile kernel (maps 0-2: many runs in one launch per step, parameters
    from each run's block in global memory) and the grouped kernel (map 4:
    parameters in the launch's constant bank) advance every run of a batch as
    the FP64 oracle advances it alone, element by element, after one and after
    three steps from random states (solid, mushy and liquid nodes; walled,
    half-periodic and periodic runs; ragged tiles)."""
    shapes = [(131, 7, 0, 0), (70, 33, 1, 0), (64, 64, 1, 1)]
    runs, orcs = [], []
    for k, (nx, ny, px, py) in enumerate(shapes):
        p = inputs.cavity(nx, ny=ny, precision=prec, periodic_x=px, periodic_y=py, L_char=100.0, Ra=1e7)
        lc = oracle_mod.lattice_config(p)
        F, G, Hm, dT = inputs.random_state(nx, ny, 5, seed=90 + k, f_base=W9.ravel(),
                                           H_range=(lc["T_fs"] - 0.3, lc["T_fl"] + lc["L_a"] + 0.3))
        dt = np.float64 if prec == 0 else np.float32
        s = lbm.Solver(p)
        s.set_state((F - W9).astype(dt), G.astype(dt), Hm.astype(dt), dT.astype(dt))
        f0, g0, h0, d0 = s.get_state()          # the oracle starts from what the solver holds
        o = oracle_mod.Oracle(p)
        o.set_state(f0.astype(np.float64) + W9, g0.astype(np.float64), h0.astype(np.float64),
                    d0.astype(np.float64))
        runs.append(s)
        orcs.append(o)
    b = lbm.Batch(runs, autotune=False).configure(64, mapping)
    for steps, margin in ((1, 1.0), (2, 2.0)):
        b.step(steps)
        for s, o in zip(runs, orcs):
            o.run(steps)
            f, g, h, d = s.get_state()
            Fo, Go, Ho, Do = o.state()
            for a, ref, name in ((f, Fo - W9, "f - w"), (g, Go, "g"), (h, Ho, "h"), (d, Do, "dT")):
                scale = max(np.abs(ref).max(), 1.0 if name == "dT" else 1e-3)
                err = np.abs(a.astype(np.float64) - ref).max() / scale
                assert err < margin * ORACLE_TOL[prec], (s.params["nx"], steps, name, err)
    b.close()
    for s in runs:
        s.close()


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("mapping", [4, 5])
def test_grouped_launches_split_large_batches(lbm, prec, mapping):
    """A batch larger than one grouped launch holds (the parameter blocks of up
    to ~40 runs fit in a launch) runs in several groups, each a chain of its
    own in the replayed graph, beside a run of 1024 x 1100 nodes (under map 4
    it keeps its own step kernel, node pairs in FP16; under map 5 it joins a
    group); every run still matches lbm_step."""
    draws = inputs.batch_draws(count=50, seed=21, n_lo=16, n_hi=48)
    draws.append(inputs.cavity(1024, ny=1100))
    runs = [lbm.Solver(dict(p, precision=prec)) for p in draws]
    solo = [lbm.Solver(dict(p, precision=prec)) for p in draws]
    b = lbm.Batch(runs, autotune=False).configure(128, mapping)
    b.step(3)
    b.step(130)
    for s in solo:
        s.step(133)
    for r, s in zip(runs, solo):
        assert r.steps == 133
        assert _same_state(r, s, mapping in EXACT_MAPS, prec)
    b.close()
    for s in runs + solo:
        s.close()


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_grouped_two_step_launches_match_the_oracle(lbm, oracle_mod, prec):
    """Map 5 (grouped launches of the two-step kernel) from random states:
    every run equals lbm_step on it bit for bit after 4 and 8 steps (two and
    four two-step launches); FP32 runs are also held to the FP64 oracle within
    FP32 rounding (4e-5 of array scale, as the single-run two-step test; the
    oracle does not round to 16 bits between steps, so FP16/BF16 runs are held
    to lbm_step only)."""
    shapes = [(131, 7, 0, 0), (70, 33, 1, 0), (64, 64, 1, 1), (3, 3, 0, 0), (300, 41, 0, 1)]
    runs, orcs, solo = [], [], []
    for k, (nx, ny, px, py) in enumerate(shapes):
        p = inputs.cavity(max(nx, ny), ny=ny, precision=prec, periodic_x=px, periodic_y=py, L_char=100.0, Ra=1e7)
        p["nx"] = nx
        lc = oracle_mod.lattice_config(p)
        F, G, Hm, dT = inputs.random_state(nx, ny, 5, seed=120 + k, f_base=W9.ravel(),
                                           H_range=(lc["T_fs"] - 0.3, lc["T_fl"] + lc["L_a"] + 0.3))
        s = lbm.Solver(p)
        s.set_state((F - W9).astype(np.float32), G.astype(np.float32), Hm.astype(np.float32), dT.astype(np.float32))
        t = lbm.Solver(p)
        t.load(s.save())
        f0, g0, h0, d0 = s.get_state()
        o = oracle_mod.Oracle(p)
        o.set_state(f0.astype(np.float64) + W9, g0.astype(np.float64), h0.astype(np.float64), d0.astype(np.float64))
        runs.append(s)
        solo.append(t)
        orcs.append(o)
    b = lbm.Batch(runs, autotune=False).configure(128, 5)
    assert b.info()["mapping"] == "grouped launches, two steps each"
    for steps in (4, 4):
        b.step(steps)
        for s, t, o in zip(runs, solo, orcs):
            t.step(steps)
            o.run(steps)
            assert s.status() == 0
            assert _same_state(s, t, True, prec)   # equal to lbm_step bit for bit
            if prec != 1:
                continue
            f, g, h, d = s.get_state()
            Fo, Go, Ho, Do = o.state()
            for a, ref, name in ((f, Fo - W9, "f - w"), (g, Go, "g"), (h, Ho, "h"), (d, Do, "dT")):
                scale = max(np.abs(ref).max(), 1.0 if name == "dT" else 1e-3)
                err = np.abs(a.astype(np.float64) - ref).max() / scale
                assert err < 4e-5, (s.params["nx"], steps, name, err)
    b.close()
    for s in runs + solo:
        s.close()


def test_map_5_gives_every_run_its_second_history(lbm):
    """Choosing map 5 allocates each run's second exchange history on the run's
    own allocator (once); FP64 batches refuse the map."""
    ps = _mixed_params(1)
    runs = [lbm.Solver(dict(p, nx=min(p["nx"], 200), ny=min(p["ny"], 200), precision=1)) for p in ps]
    b = lbm.Batch(runs, autotune=False)          # its work list comes from the first run's allocator
    before = [len(r._alloc.live) for r in runs]
    b.configure(128, 5)
    b.step(70)
    b.configure(128, 5)
    assert [len(r._alloc.live) for r in runs] == [n + 1 for n in before]
    b.close()
    for r in runs:
        r.close()
    f64 = [lbm.Solver(dict(ps[0], precision=0))]
    b = lbm.Batch(f64, autotune=False)
    with pytest.raises(lbm.LbmError):
        b.configure(128, 5)
    b.close()
    f64[0].close()
