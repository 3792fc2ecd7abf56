"""Runs the FP64 oracle to a relative KKT tolerance on the large power-law LP
(1,000,000 x 2,000,000, nnz ~ 20M) and records the iteration count and time in
``oracle/reference_runs.json``.  The benchmark's CPU-baseline leg scales its
bounded per-iteration sample by this count.  Calls only ``oracle`` and the input
generator; takes tens of minutes on one core.

usage: python oracle/run_to_tolerance.py [tol ...]
"""
import json
import os
import platform
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2508_16806_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "reference_runs.json")


def main(tols):
    lp = synth.power_law_lp()
    runs = json.load(open(OUT)) if os.path.exists(OUT) else []
    for tol in tols:
        t = time.time()
        x, y, info, trace = oracle.solve(lp, tol=tol, max_iters=200000, trace_cap=10)
        dt = time.time() - t
        runs.append(dict(workload="powerlaw 1000000x2000000 (alpha 2.1, rows 4..5000), seed 20250817",
                         nnz=lp.nnz, tol=tol, status=info["status"], iters=info["iters"],
                         attempts=info["attempts"], restarts=info["restarts"],
                         rel_gap=info["rel_gap"], rel_pres=info["rel_pres"],
                         rel_dres=info["rel_dres"], pobj=info["pobj"],
                         f_star=lp.f_star, time_s=dt, cores=1,
                         machine=platform.machine(), numpy=np.__version__))
        json.dump(runs, open(OUT, "w"), indent=1)
        print(runs[-1], flush=True)


if __name__ == "__main__":
    main([float(t) for t in sys.argv[1:]] or [1e-4])
