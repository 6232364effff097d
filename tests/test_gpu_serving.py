"""Continuous-batching serving engine (lbm_server_*).

A request's result must be the same alone and in the mix: runs admitted at
different ticks advance together in one batched launch per step.  Under map 3
(each run's own kernel) batched steps equal lbm_step bit for bit; under map 4
(the default: grouped launches) a run's steps do not depend on the other runs
in the launch, so its result equals, bit for bit, the same server's result
for the request alone.
"""
import numpy as np
import pytest

from paper_1701_00702_gb300 import inputs

pytestmark = pytest.mark.gpu
KEYS = ("melt_frac", "nu_hot", "enthalpy", "mass")


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1701_00702_gb300 import build, lbm as mod
    build.build()
    return mod


def _requests(prec, count=10, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for p in inputs.batch_draws(count=count, seed=seed, n_lo=24, n_hi=96):
        p = dict(p, precision=prec, ny=int(rng.integers(24, 97)))
        out.append((p, int(rng.integers(40, 400))))
    return out


@pytest.mark.parametrize("prec", [2, 1])
def test_each_result_is_the_same_alone_and_in_the_mix(lbm, prec):
    reqs = _requests(prec)
    srv = lbm.Server(hbm_budget_bytes=1 << 40, max_active=6, batched=True, quantum=64, precision=prec, mapping=3)
    ids = {}
    for p, n in reqs[:5]:
        ids[srv.submit(p, n)] = (p, n)
    results = []
    ticks = 0
    while len(results) < len(reqs):
        if ticks == 2:                      # later arrivals join runs already on the device
            for p, n in reqs[5:]:
                ids[srv.submit(p, n)] = (p, n)
        active, queued, _ = srv.tick()
        assert active <= 6
        results += srv.results()
        ticks += 1
        assert ticks < 10_000
    admits = sorted((r["admit_s"], r["id"]) for r in results)
    assert [i for _, i in admits] == sorted(ids)            # admitted in arrival order
    assert any(r["admit_s"] > min(q["admit_s"] for q in results) for r in results)
    for r in results:
        assert r["status"] == 0
        p, n = ids[r["id"]]
        assert r["steps"] == n
        s = lbm.Solver(p)
        s.step(n)
        d = s.diag()
        for k in KEYS:
            assert r[k] == d[k], (k, r[k], d[k])
        s.close()
    st = srv.stats()
    assert st["used_bytes"] == 0 and st["node_steps"] == sum(p["nx"] * p["ny"] * n for p, n in reqs)
    srv.close()


def test_budget_and_slots_are_respected(lbm):
    reqs = _requests(2, count=8, seed=5)
    sizes = sorted(lbm.state_bytes(p) for p, _ in reqs)
    budget = sizes[-1] + sizes[0] + sizes[1]           # the largest run fits, never all at once
    srv = lbm.Server(hbm_budget_bytes=budget, max_active=8, batched=True, quantum=32, precision=2)
    for p, n in reqs:
        srv.submit(p, n)
    done = []
    while len(done) < len(reqs):
        srv.tick()
        assert srv.stats()["used_bytes"] <= budget
        done += srv.results()
    assert srv.stats()["peak_used_bytes"] <= budget
    assert all(r["status"] == 0 for r in done)
    srv.close()


def test_plain_form_serves_one_request_at_a_time(lbm):
    reqs = _requests(1, count=4, seed=8)
    srv = lbm.Server(hbm_budget_bytes=1 << 40, max_active=8, batched=False, quantum=64, precision=1)
    for p, n in reqs:
        srv.submit(p, n)
    done = []
    while len(done) < len(reqs):
        srv.tick()
        done += srv.results()
    done.sort(key=lambda r: r["id"])
    for a, b in zip(done, done[1:]):
        assert b["admit_s"] >= a["finish_s"]
    srv.close()


def test_refused_requests(lbm):
    srv = lbm.Server(hbm_budget_bytes=1 << 20, max_active=4, batched=True, precision=2)
    with pytest.raises(lbm.LbmError):
        srv.submit(inputs.cavity(512, precision=2), 100)       # larger than the whole budget
    with pytest.raises(lbm.LbmError):
        srv.submit(inputs.cavity(16, precision=1), 100)        # another precision
    with pytest.raises(lbm.LbmError) as e:
        srv.submit(dict(inputs.cavity(16, precision=2), porosity=1.5), 100)
    assert e.value.code == -1
    srv.close()


def test_replay_of_poisson_arrivals(lbm):
    trace = inputs.serving_arrivals(count=8, rate_per_s=40.0, seed=11, grids=((64, 64), (96, 64), (128, 128)),
                                    steps_lo=200, steps_hi=2000)
    for r in trace:
        r["params"] = dict(r["params"], precision=2)
    srv = lbm.Server(hbm_budget_bytes=1 << 40, max_active=16, batched=True, quantum=128, precision=2)
    res = srv.replay(trace)
    assert len(res) == 8 and all(r["status"] == 0 for r in res)
    assert all(r["finish_s"] >= r["admit_s"] >= r["submit_s"] for r in res)
    srv.close()


@pytest.mark.parametrize("mapping", [4, 5])
def test_grouped_launches_serve_each_result_as_alone(lbm, mapping):
    """With grouped launches (map 4: every active run in one launch per step;
    map 5: two steps per launch) a request's result in the mix equals, bit for
    bit, its result when the same server configuration serves it alone."""
    reqs = _requests(2, count=8, seed=13)

    def serve(batch):
        srv = lbm.Server(hbm_budget_bytes=1 << 40, max_active=8, batched=True, quantum=64, precision=2,
                         mapping=mapping)
        ids = {srv.submit(p, n): k for k, (p, n) in enumerate(batch)}
        out = []
        while len(out) < len(batch):
            srv.tick()
            out += srv.results()
        srv.close()
        return {ids[r["id"]]: r for r in out}

    mixed = serve(reqs)
    for k, req in enumerate(reqs):
        alone = serve([req])[0]
        assert mixed[k]["status"] == 0 and alone["status"] == 0
        for key in KEYS:
            assert mixed[k][key] == alone[key], (k, key)
