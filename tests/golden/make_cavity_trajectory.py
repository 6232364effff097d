"""Writes ``cavity256_oracle_trajectory.json``: the FP64 oracle's melt
fraction, hot-wall Nusselt number, total enthalpy and mass along the full
200,000-step solve of the 256 x 256 square cavity (the Sec. IV B set-up with
porosity 0.9 and conductivity ratio 100: Ra = 1e6, Pr = 50, Da = 1e-4,
Ste = 1, H_v = 5.9, L = 256).  Fo = alpha_f t / L^2 (Eq. 54) is stored beside
each checkpoint; 200,000 steps reach Fo = 0.00153, three quarters of the
Fo = 0.002 that Sec. IV B follows.

Calls only ``oracle/``; the GPU tests compare each storage form with these
values.  Run from the repository root:

    python tests/golden/make_cavity_trajectory.py
"""
from __future__ import annotations

import json
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_1701_00702_gb300 import inputs  # noqa: E402

CHECKPOINTS = [1000, 2000, 4000, 8000, 16000, 25000, 50000, 75000, 100000, 125000, 150000, 175000, 200000]
OUT = Path(__file__).resolve().parent / "cavity256_oracle_trajectory.json"


def main() -> None:
    p = inputs.cavity(256, precision=inputs.PREC_F64)
    o = oracle.Oracle(p)
    lc = o.lc
    rows = []
    t0 = time.time()
    for k in CHECKPOINTS:
        o.run(k - o.steps)
        d = o.diag()
        rows.append(dict(steps=k, Fo=lc["alpha_f"] * k / lc["L"] ** 2, **d))
        print(f"{k:7d} steps  melt {d['melt_frac']:.8f}  Nu {d['nu_hot']:.8f}  ({time.time() - t0:.0f} s)",
              flush=True)
    OUT.write_text(json.dumps({
        "_about": "FP64 oracle along the 200,000-step solve of the 256 x 256 square cavity "
                  "(inputs.cavity(256)); written by tests/golden/make_cavity_trajectory.py, "
                  "which calls only oracle/",
        "params": p, "threads": o.threads, "rows": rows}, indent=1) + "\n")


if __name__ == "__main__":
    main()
