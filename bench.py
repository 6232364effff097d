#!/usr/bin/env python
"""Throughput of the fused three-lattice enthalpy MRT-LB step on GB300.

Prints ONE JSON line on rank 0.

Workload (default): square-cavity melting with natural convection, 256 x 256
nodes, FP32 storage, D2Q9 flow + D2Q5 PCM + D2Q5 metal lattices, Ra = 1e6,
Pr = 50, Da = 1e-4, porosity 0.9, Ste = 1, conductivity ratio 100,
H_v = 5.9, hot left / cold right walls, adiabatic top and bottom.  One
benchmark step advances the run by ``--lb-steps`` time steps (a chunk of the
200k-step solve); L2 is flushed between benchmark steps.  The metric is MLUPS
(million node updates per second, every node counted).  The run takes the
library's automatic step form: two time steps per launch at 256 x 256.

Besides the headline number the line carries:
  * roofline: the one-step kernel (one node per thread, one step per launch)
    on the 2048 x 2048 cavity (0.7 GB of state, far beyond L2), algorithmic
    160 B per node update (19 FP32 populations and the exchange history, each
    read and written once) against the measured HBM copy bandwidth;
  * two_step: the automatic form on that cavity, two steps per launch (the
    state crosses HBM once per two node updates);
  * e2e: the same workload through the C ABI with host buffers: each step
    uploads the full state from pinned memory, advances it and reads back
    T_f, T_s, f_l, u_x, u_y;
  * cpu_baseline: the FP64 oracle timed on this host's cores on a bounded
    sample of the same cavity.

``--impl reference`` times the oracle alone on the same workload.
With torchrun (N > 1) every rank runs its own cavity (independent runs, weak
scaling); no data crosses ranks, only the timing maximum.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "coupled MRT-LB MLUPS (fused three-lattice step)"
UNIT = "MLUPS"
L2_FLUSH_BYTES = 512 << 20


PREC_NAMES = {0: "f64", 1: "f32", 2: "f16", 3: "bf16"}
FORM_NAMES = {1: "one node per thread", 2: "node pairs", 3: "two steps per launch"}


def launches_per_call(form: int, nsteps: int) -> int:
    """Kernel launches of one lbm_step(nsteps) call from state copy 0 with an
    even nsteps: 64-step graphs (32 launches each in the two-step form), then
    pairs of two-step launches for 4 steps each, then single steps."""
    if form != 3:
        return nsteps
    graphs, rest = divmod(nsteps, 64)
    return graphs * 32 + (rest // 4) * 2 + rest % 4


def bytes_per_update(qt: int, flow: int, precision: int) -> int:
    """Algorithmic HBM bytes per node update: every population the method
    stores read and written once, plus the exchange history of Remark III.
    FP64: 8-byte populations and history; FP32: 4-byte; FP16/BF16: 2-byte
    populations with an FP32 history.  D2Q9 flow + D2Q5 + D2Q5 gives 320, 160
    and 84 B."""
    fl = 9 if flow else 0
    if precision == 0:
        return (fl + 2 * qt + 1) * 8 * 2
    if precision == 1:
        return (fl + 2 * qt + 1) * 4 * 2
    return (fl + 2 * qt) * 2 * 2 + 4 * 2


def stored_bytes_per_update(qt: int, flow: int, precision: int) -> int:
    """Bytes the implementation moves per node update: the algorithmic bytes
    plus its own extra planes -- FP32 keeps the low part of the float-float
    PCM rest population (one more FP32 plane), FP16/BF16 keep both thermal
    rest populations in FP32 (two 16-bit planes become FP32)."""
    b = bytes_per_update(qt, flow, precision)
    if precision == 1:
        return b + 4 * 2
    if precision in (2, 3):
        return b + 2 * 2 * 2
    return b


# DRAM traffic of one launch of the roofline kernel (fused_step, FP32, D2Q5,
# flow, 2048 x 2048 cavity) and of the two-step kernel on the same cavity:
# dram__bytes_read.sum + dram__bytes_write.sum from one ncu capture each,
# taken for the kernel sources whose code hash is given; the bench reports
# them only while the sources still hash to that value.
ROOFLINE_TRAFFIC = {
    "bytes_per_launch": 352022528 + 299681280,
    "kernel_sources_sha256_16": "927ee769a50e6f38",
    "gpu__dram_throughput_pct": 84.2,
    "captured": "2026-12-04, ncu --set full --clock-control none, one launch after two "
                "(profiles/fused_step_cavity2048_fp32.md)",
}
TWO_STEP_TRAFFIC = {
    "bytes_per_launch": 352046080 + 305852160,
    "kernel_sources_sha256_16": "927ee769a50e6f38",
    "gpu__dram_throughput_pct": 51.1,
    "captured": "2026-12-04, ncu --set full --clock-control none, one launch after two "
                "(profiles/fused_step2_cavity2048_fp32.md)",
}


def measured_traffic(n: int, table: dict = ROOFLINE_TRAFFIC):
    """ncu DRAM bytes per launch from `table`, or None for another grid size
    or once the kernel sources have changed since the capture."""
    if n != 2048 or kernel_sources_hash() != table["kernel_sources_sha256_16"]:
        return None
    return table["bytes_per_launch"]


def kernel_sources_hash() -> str:
    """First 16 hex digits of the sha256 of the step kernels' sources with
    // comments, trailing blanks and empty lines removed (a comment edit does
    not invalidate a capture; any code change does)."""
    h = hashlib.sha256()
    for name in ("lbm_kernels.cuh", "lbm_launch.cuh", "lbm_kernels_f32.cu"):
        text = (ROOT / "paper_1701_00702_gb300" / "csrc" / name).read_text()
        code = [ln.split("//", 1)[0].rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in code if ln).encode())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="cavity side")
    ap.add_argument("--precision", default="f32", choices=["f64", "f32", "f16", "bf16"],
                    help="storage form of the headline run")
    ap.add_argument("--lb-steps", type=int, default=20000,
                    help="LB time steps per benchmark step (a tenth of the 200k-step solve)")
    ap.add_argument("--roofline-n", type=int, default=2048)
    ap.add_argument("--step-form", default="auto", choices=["auto", "single", "pairs", "two"],
                    help="step form of the headline run (lbm_set_step_form; auto: the library's choice)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-runs", type=int, default=64)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=16)
    ap.add_argument("--serve-step-scale", type=float, default=0.1,
                    help="scale of the serving trace's step counts (log-uniform 1e4..5e5 before scaling)")
    ap.add_argument("--serve-full", action="store_true",
                    help="serve the stated trace (>= 64 requests, 1e4..5e5 steps) and add a run under a "
                         "budget that binds (several minutes)")
    ap.add_argument("--serve-tight-budget-gb", type=float, default=0.5)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int) -> float:
    """The largest of every rank's x (the slowest rank's time); x itself at N = 1."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_mlups(world: int, cells: int, lb_steps: int, steps: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas, each updating `cells` nodes
    `lb_steps` times per benchmark step for `steps` steps, over the slowest
    rank's `seconds`."""
    return world * cells * lb_steps * steps / seconds / 1e6


def workload_config(args, p, chunk):
    return {
        "workload": f"square-cavity melting with natural convection {p['nx']}x{p['ny']} {PREC_NAMES[p['precision']].upper()}",
        "grid": [p["nx"], p["ny"]],
        "lattices": "D2Q9 flow + D2Q5 PCM + D2Q5 metal",
        "Ra": p["Ra"], "Pr": p["Pr"], "Da": p["Da"], "porosity": p["porosity"], "Ste": p["Ste"],
        "cond_ratio": p["cond_ratio"], "Nu_i": p["Nu_i"],
        "lb_steps_per_step": chunk,
        "l2": "flushed (512 MB write) between timed steps; within a step the state stays on chip as in a real solve",
        "parallelism": "independent runs per GPU",
    }


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "50"]
            if self.bus_id:
                cmd += ["-i", self.bus_id]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            # the timed region starts only once the sampler is running
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 2.0 and self.proc.poll() is None:
                if Path(self.path).stat().st_size > 0:
                    break
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in Path(self.path).read_text().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 10:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def time_oracle(p: dict, budget_s: float, max_steps: int):
    """Times the FP64 oracle on cavity p for about budget_s seconds of CPU work."""
    import oracle
    o = oracle.Oracle(p)
    o.run(1)                                  # starts the thread pool
    t0 = time.perf_counter()
    o.run(2)
    per = max((time.perf_counter() - t0) / 2.0, 1e-6)
    n = int(max(2, min(max_steps, budget_s / per)))
    t0 = time.perf_counter()
    o.run(n)
    dt = time.perf_counter() - t0
    per = dt / n
    cells = p["nx"] * p["ny"]
    out = {"value": cells * n / dt / 1e6, "unit": UNIT, "cores": o.threads, "kind": "oracle",
           "sample": f"{n} time steps of the {p['nx']}x{p['ny']} cavity from the uniform start "
                     f"({dt:.1f} s, FP64 oracle, OpenMP over rows)"}
    cores = o.threads
    # one thread on the same cavity, then the 200 x 4 conduction case in full (20,000 steps)
    o1 = oracle.Oracle(p, threads=1)
    n1 = int(max(2, min(max_steps, budget_s / 4.0 / (per * cores))))
    t0 = time.perf_counter()
    o1.run(n1)
    d1 = time.perf_counter() - t0
    out["single_thread"] = {"value": cells * n1 / d1 / 1e6, "unit": UNIT,
                            "sample": f"{n1} time steps of the same cavity on one thread ({d1:.1f} s)"}
    oracle.lib().orc_set_threads(cores)
    from paper_1701_00702_gb300 import inputs
    oc = oracle.Oracle(inputs.conduction_1d())
    t0 = time.perf_counter()
    oc.run(20_000)
    out["conduction_200x4_20000_steps_s"] = time.perf_counter() - t0
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1701_00702_gb300 import inputs
    p = inputs.cavity(args.n, precision=1)
    import oracle
    o = oracle.Oracle(p)
    t0 = time.perf_counter()
    o.run(2)
    per = max((time.perf_counter() - t0) / 2.0, 1e-6)
    total = args.steps + args.warmup
    per_step = int(max(1, min(args.lb_steps, 150.0 / total / per)))
    for _ in range(args.warmup):
        o.run(per_step)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.run(per_step)
        times.append(time.perf_counter() - t0)
    cells = p["nx"] * p["ny"]
    value = cells * per_step * len(times) / sum(times) / 1e6
    cfg = workload_config(args, p, args.lb_steps)
    cfg["reference_lb_steps_per_step"] = per_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": o.threads, "kind": "oracle",
                         "sample": f"{per_step} time steps of the {p['nx']}x{p['ny']} cavity per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def bench_serving(args, lbm, inputs, stream, plain_mlups: float, seed: int = 1701):
    """Poisson arrivals of melting runs (grids 128^2, 256^2, 512^2, 1024^2,
    2048x1024; mixed porosity, Da, Ra, Ste; step counts log-uniform over the
    trace's range) at ~80 % of the plain form's capacity, served by the plain
    form (FP32, one request at a time in arrival order) and by continuous
    batching (FP16) under the 150 GB HBM budget and, with --serve-full, under
    a budget small enough to bind; every form replays the same trace on the
    host clock."""
    import numpy as np
    scale = 1.0 if args.serve_full else args.serve_step_scale
    count = max(64, args.serve_requests) if args.serve_full else args.serve_requests
    lo, hi = int(1e4 * scale), int(5e5 * scale)
    grids = ((128, 128), (256, 256), (512, 512), (1024, 1024), (2048, 1024))
    mean_nodes = float(np.mean([a * b for a, b in grids]))
    mean_steps = (hi - lo) / np.log(hi / lo)
    capacity = plain_mlups * 1e6 / (mean_nodes * mean_steps)   # requests per second of the plain form, roughly
    rate = 0.8 * capacity
    base = inputs.serving_arrivals(count=count, rate_per_s=rate, seed=seed, grids=grids,
                                   steps_lo=lo, steps_hi=hi)
    out = {"requests": len(base), "arrival_rate_per_s": rate, "step_range": [lo, hi],
           "note": ("the stated trace: 10k..500k steps" if scale == 1.0 else
                    f"step counts of the 1e4..5e5 serving trace scaled by {scale}"), "forms": []}
    # (name, batched, precision, HBM budget GB, arrival-rate factor)
    forms = [("plain FP32 (one at a time)", False, 1, 150.0, 1.0), ("continuous batching FP16", True, 2, 150.0, 1.0)]
    if args.serve_full:
        forms += [("continuous batching FP16, tight budget", True, 2, args.serve_tight_budget_gb, 1.0),
                  ("plain FP32 (one at a time), arrivals at 2x its capacity", False, 1, 150.0, 2.5),
                  ("continuous batching FP16, arrivals at 2x the plain capacity", True, 2, 150.0, 2.5)]
    for name, batched, prec, budget_gb, speed in forms:
        # the same requests; a factor > 1 compresses their arrival times (0.8 x 2.5 = 2x capacity)
        trace = [dict(r, arrival_s=r["arrival_s"] / speed, params=dict(r["params"], precision=prec)) for r in base]
        srv = lbm.Server(hbm_budget_bytes=int(budget_gb * 1e9), max_active=64, batched=batched, quantum=256,
                         precision=prec, stream=stream)
        res = srv.replay(trace)
        st = srv.stats()
        srv.close()
        lat = np.array([r["finish_s"] - r["submit_s"] for r in res])
        wait = np.array([r["admit_s"] - r["submit_s"] for r in res])
        span = max(r["finish_s"] for r in res) - min(r["submit_s"] for r in res)
        out["forms"].append({
            "form": name, "ok": all(r["status"] == 0 for r in res), "hbm_budget_gb": budget_gb,
            "arrival_rate_per_s": rate * speed,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "p50_queue_s": float(np.percentile(wait, 50)), "max_queue_s": float(wait.max()),
            "runs_per_s": len(res) / span, "aggregate_mlups": st["node_steps"] / span / 1e6,
            "busy_mlups": st["node_steps"] / max(st["busy_s"], 1e-9) / 1e6,
            "peak_admitted_gb": st["peak_used_bytes"] / 1e9})
    return out


TRAJECTORY = ROOT / "tests" / "golden" / "cavity256_oracle_trajectory.json"


def accuracy_forms():
    """(name, precision, batched) of every form whose error the bench reports."""
    return (("f64", 0, False), ("f32", 1, False), ("f16", 2, False), ("bf16", 3, False),
            ("f16 batched (map 3, with three other cavities)", 2, True))


def bench_accuracy(args, lbm, inputs, stream) -> dict | None:
    """Error of each storage form against the FP64 oracle over the full
    200,000-step solve of the 256 x 256 cavity (to Fo = 0.00153): melt
    fraction and hot-wall Nusselt number at every checkpoint of the stored
    oracle trajectory (tests/golden/cavity256_oracle_trajectory.json, written
    by a script that runs only the oracle).  The batched form advances the
    cavity in a map-3 batch beside three other cavities."""
    if args.n != 256 or not TRAJECTORY.exists():
        return None
    ref = json.loads(TRAJECTORY.read_text())
    rows = ref["rows"]
    out = {"workload": "256x256 cavity, full 200,000-step solve", "reference": "FP64 oracle (stored trajectory)",
           "checkpoints": [r["steps"] for r in rows], "Fo": [r["Fo"] for r in rows],
           "melt_frac": [r["melt_frac"] for r in rows], "nu_hot": [r["nu_hot"] for r in rows], "forms": []}
    for name, prec, batched in accuracy_forms():
        s = lbm.Solver(inputs.cavity(256, precision=prec), stream=stream)
        others, b = [], None
        if batched:
            others = [lbm.Solver(dict(q, precision=prec), stream=stream)
                      for q in inputs.batch_draws(count=3, seed=5, n_lo=64, n_hi=160)]
            b = lbm.Batch([s] + others, autotune=False, stream=stream).configure(128, 3)
        em, en = [], []
        for row in rows:
            k = row["steps"] - s.steps
            if b is not None:
                b.step(k)
            else:
                s.step(k)
            d = s.diag()
            em.append(abs(d["melt_frac"] / row["melt_frac"] - 1.0))
            en.append(abs(d["nu_hot"] / row["nu_hot"] - 1.0))
        ok = s.status() == 0
        if b is not None:
            b.close()
        for r in [s] + others:
            r.close()
        out["forms"].append({"form": name, "ok": ok, "melt_frac_rel_err": em, "nu_hot_rel_err": en,
                             "max_melt_frac_rel_err": max(em), "max_nu_hot_rel_err": max(en)})
    return out


def bench_batched(args, lbm, inputs, torch, stream, steps_per_solve: int = 10_000, chunk: int = 64, reps: int = 3):
    """64 cavities, sides uniform in [64, 512], porosity, Da, Ra, Ste drawn as in
    the batched workload; every form advances all runs by the same steps."""
    draws = inputs.batch_draws(count=args.batch_runs)
    nodes = sum(p["nx"] * p["ny"] for p in draws)

    def make(prec):
        return [lbm.Solver(dict(p, precision=prec), stream=stream) for p in draws]

    def timed(fn):
        fn()
        stream.synchronize()
        e = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in e:
            a.record(stream)
            fn()
            b.record(stream)
        stream.synchronize()
        return sum(a.elapsed_time(b) for a, b in e) / (reps * chunk)   # ms per step of all runs

    out = {"runs": len(draws), "nodes": nodes, "steps_per_solve": steps_per_solve, "forms": []}
    runs = make(1)
    ms = timed(lambda: [r.step(chunk) for r in runs])
    ok = all(r.status() == 0 for r in runs)
    for r in runs:
        r.close()
    out["forms"].append({"form": "plain per-run FP32", "ms_per_step": ms, "mlups": nodes / (ms / 1e3) / 1e6,
                         "solves_per_s": len(draws) / (ms / 1e3 * steps_per_solve), "ok": ok})
    for prec, name in ((1, "batched FP32"), (2, "batched FP16")):
        runs = make(prec)
        b = lbm.Batch(runs, autotune=True, stream=stream)
        ms = timed(lambda: b.step(chunk))
        info = b.info()
        if info["mapping"] == "single-run kernel chains":
            shapes = {}
            for bx, by in b.blocks():
                shapes[f"{bx}x{by}"] = shapes.get(f"{bx}x{by}", 0) + 1
            info["block_shapes"] = shapes
        ok = all(r.status() == 0 for r in runs)
        b.close()
        for r in runs:
            r.close()
        out["forms"].append({"form": name, "ms_per_step": ms, "mlups": nodes / (ms / 1e3) / 1e6,
                             "solves_per_s": len(draws) / (ms / 1e3 * steps_per_solve), "ok": ok,
                             "tuned": info})
    base = out["forms"][0]["solves_per_s"]
    for f in out["forms"]:
        f["speedup_vs_plain_fp32"] = f["solves_per_s"] / base
    return out

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    from paper_1701_00702_gb300 import build, inputs, lbm
    build.build()

    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    chunk = args.lb_steps
    prec = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}[args.precision]
    p = inputs.cavity(args.n, precision=prec)
    cells = p["nx"] * p["ny"]
    want_form = {"auto": 0, "single": 1, "pairs": 2, "two": 3}[args.step_form]
    form = lbm.step_form_for(p, want_form)
    bpu = bytes_per_update(p["thermal_q"], p["flow"], p["precision"])
    props = torch.cuda.get_device_properties(dev)
    bus = getattr(props, "pci_bus_id", None)
    bus_id = None
    if bus is not None:
        bus_id = f"{getattr(props, 'pci_domain_id', 0):08X}:{bus:02X}:{getattr(props, 'pci_device_id', 0):02X}.0"

    with torch.cuda.stream(stream):
        s = lbm.Solver(p, stream=stream).set_step_form(want_form)
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        for _ in range(args.warmup):
            s.step(chunk)
            flush.zero_()
        stream.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clocks = ClockSampler(bus_id)
        clocks.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize(dev)
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            s.step(chunk)
            b.record(stream)
        stream.synchronize()
        torch.cuda.synchronize(dev)
        times_ms = [a.elapsed_time(b) for a, b in ev]
        clk = clocks.stop()
        if s.status() != 0:
            raise SystemExit("solver reported an unstable state")
        total_ms = max_over_ranks(sum(times_ms), world)
        value = replica_mlups(world, cells, chunk, args.steps, total_ms / 1e3)
        launch_ms_small = total_ms / (args.steps * chunk)

        # end to end through the C ABI with host buffers
        e2e = None
        if not args.no_e2e:
            f0, g0, h0, d0 = s.get_state()
            tdt = torch.float64 if prec == 0 else torch.float32
            pin = {k: torch.empty(a.shape, dtype=tdt, pin_memory=True).numpy()
                   for k, a in (("f", f0), ("g", g0), ("h", h0), ("dT", d0))}
            for k, a in (("f", f0), ("g", g0), ("h", h0), ("dT", d0)):
                pin[k][...] = a
            outs = {name: torch.empty((p["ny"], p["nx"]), dtype=tdt, pin_memory=True).numpy()
                    for name in ("T_f", "T_s", "f_l", "u_x", "u_y")}
            h2d = sum(a.nbytes for a in pin.values())
            d2h = sum(a.nbytes for a in outs.values())
            for _ in range(max(1, args.warmup)):
                s.set_state(pin["f"], pin["g"], pin["h"], pin["dT"])
                s.step(chunk)
                s.fields_into(outs)
            if world > 1:
                torch.distributed.barrier()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                s.set_state(pin["f"], pin["g"], pin["h"], pin["dT"])
                s.step(chunk)
                s.fields_into(outs)
            e2e_s = max_over_ranks(time.perf_counter() - t0, world)
            e2e = {"value": replica_mlups(world, cells, chunk, args.steps, e2e_s), "unit": UNIT,
                   "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
        s.close()
        del flush

        def time_form(prec: int, n: int, per: int, reps: int = 3, step_form: int = 0):
            pf = inputs.cavity(n, precision=prec)
            sf = lbm.Solver(pf, stream=stream).set_step_form(step_form)
            sf.step(64)
            stream.synchronize()
            e = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for a, b in e:
                a.record(stream)
                sf.step(per)
                b.record(stream)
            stream.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in e) / (reps * per)
            rc = sf.status()
            sf.close()
            if rc != 0:
                raise SystemExit(f"form {PREC_NAMES[prec]} {n}^2 reported an unstable state")
            return ms

        # roofline: the one-step kernel on a state far larger than L2
        roof, two_step = None, None
        if args.roofline_n > 0:
            pr = inputs.cavity(args.roofline_n, precision=1)
            ms = time_form(1, args.roofline_n, 128, step_form=1)
            peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) if (ROOT / "MEASURED_PEAKS.json").exists() else {}
            peak = float(peaks.get("hbm_gbs", 6800.0))
            nodes = pr["nx"] * pr["ny"]
            b_alg = bytes_per_update(pr["thermal_q"], pr["flow"], 1)
            b_sto = stored_bytes_per_update(pr["thermal_q"], pr["flow"], 1)
            achieved = b_alg * nodes / (ms / 1e3) / 1e9
            traffic = measured_traffic(pr["nx"])
            roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic,
                    "kernel": "fused_step<float, Q_T=5, flow> (one node per thread, one step per launch)",
                    "workload": f"square-cavity melting {pr['nx']}x{pr['ny']} FP32 (state {lbm.state_bytes(pr) / 2**30:.2f} GiB)",
                    "bytes_per_update": b_alg,
                    "bytes_basis": "algorithmic: 19 FP32 populations and the FP32 exchange history, each read and "
                                   "written once (D2Q9 flow + D2Q5 PCM + D2Q5 metal)",
                    "overhead_bytes_per_update": b_sto - b_alg,
                    "overhead": "the low part of the float-float PCM rest population, read and written once",
                    "units_per_launch": nodes,
                    "mlups": nodes / (ms / 1e3) / 1e6, "avg_launch_us": ms * 1e3,
                    "peak_kind": "measured copy bandwidth (STREAM-style copy, read + write bytes), not the HBM "
                                 "data-sheet rate",
                    "peak_source": "measured" if peaks else "fallback",
                    "traffic_source": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum, {ROOFLINE_TRAFFIC['captured']}"
                                       if traffic else "no capture of the current kernel sources"),
                    "ncu_gpu__dram_throughput_pct": ROOFLINE_TRAFFIC["gpu__dram_throughput_pct"] if traffic else None}
            # the automatic form on the same cavity: two steps per launch, the state
            # through HBM once per launch
            ms2 = time_form(1, args.roofline_n, 128)
            t2 = measured_traffic(pr["nx"], TWO_STEP_TRAFFIC)
            launch_s = 2 * ms2 / 1e3
            two_step = {"kernel": "fused_step2<float, Q_T=5, flow> (blocks of 34 x 12 threads, inner tiles 32 x 10)",
                        "step_form": FORM_NAMES[lbm.step_form_for(pr, 0)],
                        "workload": roof["workload"], "us_per_step": ms2 * 1e3, "avg_launch_us": launch_s * 1e6,
                        "mlups": nodes / (ms2 / 1e3) / 1e6, "speedup_over_one_step": ms / ms2,
                        "hbm_bytes_per_launch_algorithmic": b_alg * nodes,
                        "hbm_basis": "the state read and written once per launch (two node updates): 160 B per "
                                     "node per launch, 80 B per node update",
                        "gbs_hbm_algorithmic": b_alg * nodes / launch_s / 1e9,
                        "frac_of_measured_hbm": b_alg * nodes / launch_s / 1e9 / peak,
                        "gbs_per_update_basis": b_alg * nodes / (ms2 / 1e3) / 1e9,
                        "per_update_basis_note": "160 B per node update over the per-step time: the one-step "
                                                 "kernel's roofline quantity, above the copy bandwidth because "
                                                 "two updates share one HBM round trip",
                        "traffic": t2,
                        "traffic_source": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum, {TWO_STEP_TRAFFIC['captured']}"
                                           if t2 else "no capture of the current kernel sources"),
                        "bound": "instruction issue (the ring's redundant updates and both steps' arithmetic), "
                                 "not HBM"}

        # many unequal cavities: plain per-run FP32 vs one launch per step for all runs
        batched = None
        if not args.no_batched:
            batched = bench_batched(args, lbm, inputs, torch, stream)

        serving = None
        if not args.no_serving:
            # the plain form's speed on large runs: its automatic form (two steps per launch in FP32)
            plain = two_step["mlups"] if two_step else (roof["mlups"] if roof else 30000.0)
            serving = bench_serving(args, lbm, inputs, stream, plain)

        accuracy = None if args.no_accuracy else bench_accuracy(args, lbm, inputs, stream)

        # every storage form of the same step, on the L2-resident and the HBM-bound cavity
        forms = []
        if args.roofline_n > 0:
            peak = roof["peak"]
            for fprec in (1, 2, 3):
                for n, per in ((args.roofline_n, 128), (args.n, 2048)):
                    ms = time_form(fprec, n, per)
                    b = bytes_per_update(5, 1, fprec)
                    gbs = b * n * n / (ms / 1e3) / 1e9
                    ff = lbm.step_form_for(inputs.cavity(n, precision=fprec), 0)
                    # two steps per launch: the state crosses HBM once per two updates
                    crossing = b / 2 if ff == 3 else b
                    forms.append({"precision": PREC_NAMES[fprec], "grid": n, "step_form": FORM_NAMES[ff],
                                  "us_per_step": ms * 1e3,
                                  "mlups": n * n / (ms / 1e3) / 1e6, "bytes_per_update": b,
                                  "overhead_bytes_per_update": stored_bytes_per_update(5, 1, fprec) - b,
                                  "gbs_algorithmic": gbs, "hbm_bytes_per_update_crossing": crossing,
                                  "frac_of_measured_hbm": crossing * n * n / (ms / 1e3) / 1e9 / peak})

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu:
        cpu = time_oracle(p, budget_s=12.0, max_steps=chunk)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": PREC_NAMES[prec], "data": "synthetic",
        "config": workload_config(args, p, chunk),
        "roofline": roof,
        "two_step": two_step,
        "l2_resident": {"step_form": FORM_NAMES[form], "us_per_step": launch_ms_small * 1e3,
                        "avg_launch_us": launch_ms_small * 1e3 * chunk / launches_per_call(form, chunk),
                        "gbs_algorithmic_per_update_basis": bpu * cells / (launch_ms_small / 1e3) / 1e9,
                        "bytes_per_update": bpu,
                        "note": f"{p['nx']}x{p['ny']} state is L2-resident; launch-to-launch time inside CUDA graphs"},
        "forms": forms if args.roofline_n > 0 else None,
        "accuracy": accuracy,
        "batched": batched,
        "serving": serving,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps * launches_per_call(form, chunk),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
