"""Whole solves on the GPU against the FP64 oracle.

* The 256 x 256 square cavity (Sec. IV B set-up, porosity 0.9, conductivity
  ratio 100, Ra = 1e6) for its full 200,000 steps (Fo = 0.00153), in every
  storage form and inside a map-3 batch: melt fraction and hot-wall Nusselt
  number at each checkpoint of the stored oracle trajectory
  (``tests/golden/cavity256_oracle_trajectory.json``, written by a script
  that runs only the oracle).  Tolerances: FP64 1e-9 (rounding), FP32 1e-4,
  FP16 1e-3 (the method's stated target for the mixed form, over the whole
  solve); BF16 keeps 8 significant bits and is held to 2e-2 only -- it does
  not meet the 1e-3 target.
* The 1024 x 1024 cavity for 100,000 steps: the 16-bit forms against FP32.
* The differentially heated cavity (the walled cavity with flow in its
  natural-convection limit): steady hot-wall Nusselt number of the GPU path
  against the oracle's and against the published benchmark.
"""
import json
from pathlib import Path

import numpy as np
import pytest

from paper_1701_00702_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = Path(__file__).parent / "golden"
TRAJ = json.loads((GOLDEN / "cavity256_oracle_trajectory.json").read_text())
DVD = {row["Ra"]: row["Nu_mean"] for row in json.loads((GOLDEN / "de_vahl_davis_1983.json").read_text())["rows"]}

# relative error bound on melt fraction and hot-wall Nu, per storage form
FULL_SOLVE_TOL = {0: 1e-9, 1: 1e-4, 2: 1e-3, 3: 2e-2}


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1701_00702_gb300 import build, lbm as mod
    build.build()
    return mod


def _trajectory_errors(lbm, prec, batched):
    s = lbm.Solver(inputs.cavity(256, precision=prec))
    others, b = [], None
    if batched:
        others = [lbm.Solver(dict(q, precision=prec)) for q in inputs.batch_draws(count=3, seed=5, n_lo=64, n_hi=160)]
        b = lbm.Batch([s] + others, autotune=False).configure(128, 3)
    errs = []
    for row in TRAJ["rows"]:
        k = row["steps"] - s.steps
        if b is not None:
            b.step(k)
        else:
            s.step(k)
        assert s.status() == 0
        d = s.diag()
        errs.append((row["steps"], abs(d["melt_frac"] / row["melt_frac"] - 1.0),
                     abs(d["nu_hot"] / row["nu_hot"] - 1.0)))
    if b is not None:
        b.close()
    for r in [s] + others:
        r.close()
    return errs


@pytest.mark.parametrize("prec,batched", [(0, False), (1, False), (2, False), (3, False), (2, True)])
def test_full_200k_step_solve_against_the_oracle(lbm, prec, batched):
    assert TRAJ["rows"][-1]["steps"] == 200000 and TRAJ["params"]["nx"] == 256
    tol = FULL_SOLVE_TOL[prec]
    for steps, em, en in _trajectory_errors(lbm, prec, batched):
        assert em < tol and en < tol, (steps, em, en)


# 1024 x 1024 against FP32 (melt fraction, hot-wall Nu).  FP16 stays within
# 1e-3 of FP32 in melt fraction over the first 100,000 steps; its Nusselt number
# also stays within 1e-3 except near the instants when a new column of nodes
# starts to melt early in the solve (the melting range T_fs..T_fl is 0.002
# wide, so each column melts as a discrete event and a few steps of delay move
# the wall flux for a moment): at most 1.56e-3, at 20,000 steps (Fo = 1e-5).
# BF16: up to 1.8e-2.
GRID1024_TOL = {2: (1e-3, 2e-3), 3: (2e-2, 2e-2)}   # (melt fraction, Nu)


@pytest.mark.parametrize("prec", [2, 3])
def test_1024_cavity_100k_steps_against_fp32(lbm, prec):
    """The 1024 x 1024 cavity (the mixed-precision workload's size): melt
    fraction and hot-wall Nusselt number of the 16-bit form against the FP32
    path every 10,000 steps up to 100,000."""
    tol_m, tol_n = GRID1024_TOL[prec]
    runs = {q: lbm.Solver(inputs.cavity(1024, precision=q)) for q in (1, prec)}
    for k in range(10):
        d = {}
        for q, s in runs.items():
            s.step(10000)
            assert s.status() == 0
            d[q] = s.diag()
        em = abs(d[prec]["melt_frac"] / d[1]["melt_frac"] - 1)
        en = abs(d[prec]["nu_hot"] / d[1]["nu_hot"] - 1)
        assert em < tol_m and en < tol_n, ((k + 1) * 10000, em, en)
    for s in runs.values():
        s.close()


def _steady_nu(run_steps, diag, chunk=2000, max_steps=60000, rtol=2e-6):
    prev, done = None, 0
    while done < max_steps:
        run_steps(chunk)
        done += chunk
        nu = diag()["nu_hot"]
        if prev is not None and abs(nu - prev) < rtol * abs(nu):
            return nu, done
        prev = nu
    raise AssertionError(f"no steady state within {max_steps} steps")


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-5)])
def test_heated_cavity_matches_the_oracle_and_the_benchmark(lbm, oracle_mod, prec, tol):
    """64 x 64, Ra = 1e5: the walls, corners and buoyancy-driven flow of the GPU
    path give the oracle's steady Nusselt number, within 2 % of the benchmark."""
    p = inputs.heated_cavity(64, 1e5, precision=prec)
    s = lbm.Solver(p)
    nu, steps = _steady_nu(s.step, s.diag)
    o = oracle_mod.Oracle(inputs.heated_cavity(64, 1e5)).run(steps)
    assert abs(nu / o.diag()["nu_hot"] - 1.0) < tol
    assert abs(nu / DVD[1e5] - 1.0) < 0.02
    s.close()


@pytest.mark.parametrize("Ra,k_f", [(1e3, 0.2), (1e4, 0.05), (1e5, 0.1)])
def test_heated_cavity_128_within_one_percent_of_the_benchmark(lbm, Ra, k_f):
    s = lbm.Solver(inputs.heated_cavity(128, Ra, k_f=k_f, precision=1))
    nu, _ = _steady_nu(s.step, s.diag, chunk=4000, max_steps=200000)
    assert abs(nu / DVD[Ra] - 1.0) < 0.01, (Ra, nu)
    s.close()
