"""Batched stepping of unequal cavities in one launch per time step.

A batched step must equal lbm_step on each run bit for bit (the per-node
arithmetic is shared), under every tile-width cap and cell-to-block map.
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
    for x, y in zip(batch_runs, solo):
        assert x.steps == y.steps == 153
        assert np.array_equal(x.save(), y.save())
    b.close()
    for s in batch_runs + solo:
        s.close()


def test_every_map_gives_the_same_state(lbm):
    ps = _mixed_params(1)
    ref = [lbm.Solver(p) for p in ps]
    for s in ref:
        s.step(40)
    want = [s.save() for s in ref]
    for cap in (32, 64, 128, 256):
        for mapping in (0, 1, 2, 3):
            runs = [lbm.Solver(p) for p in ps]
            b = lbm.Batch(runs, autotune=False).configure(cap, mapping)
            b.step(40)
            for r, w in zip(runs, want):
                assert np.array_equal(r.save(), w), (cap, mapping)
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
        assert np.array_equal(r.save(), t.save())
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
