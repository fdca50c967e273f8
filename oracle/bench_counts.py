"""Writes oracle/bench_counts.json: the step counts of the oracle's own full two-grid
solve of each benchmark workload (coarse GMRES-DR cycles and Arnoldi steps, fine-grid
operator products and cycles).  The benchmark's CPU-baseline arm times bounded pieces of
the oracle and scales them to one solve with these counts.

TEST INFRASTRUCTURE ONLY: calls nothing but oracle/ and tg_inputs.
Usage: python -m oracle.bench_counts [workload ...]   (takes tens of minutes for cd3d_255)
"""
import json
import os
import sys
import time

import numpy as np

import tg_inputs as gi
from oracle import krylov, twogrid
from oracle.operators import CD2D, CD3D, Operator

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "bench_counts.json")

# the same parameters as the benchmark's workloads (bench.py WORKLOADS)
WORKLOADS = {
    "cd3d_255": dict(kind=CD3D, N=255, beta=(2.0, 1.0, 0.5), m=60, k=30, nev=30, rtolev=1e-2, rtol_c=1e-8,
                     rtol=1e-8, ncyc=20, restart_mvps=None),
    "cd2d_127": dict(kind=CD2D, N=127, beta=(1.0,), m=30, k=15, nev=15, rtolev=1e-4, rtol_c=1e-8,
                     rtol=1e-8, ncyc=0, restart_mvps=60),
}


def run(name):
    w = WORKLOADS[name]
    op = Operator(w["kind"], w["N"], w["beta"])
    b = gi.rhs(op.n, 0)
    t0 = time.time()
    res = twogrid.two_grid_solve(op, b, m=w["m"], k=w["k"], nev=w["nev"], rtolev=w["rtolev"],
                                 rtol_c=w["rtol_c"], method="bicgstab", proj="minres", rtol=w["rtol"],
                                 ncyc=w["ncyc"], restart_mvps=w["restart_mvps"])
    return {"coarse_cycles": res.coarse.cycles, "coarse_steps": res.coarse.mvps,
            "fine_mvps": res.solve.mvps, "fine_cycles": res.solve.cycles,
            "relres": res.solve.relres, "converged": bool(res.solve.converged),
            "oracle_seconds": round(time.time() - t0, 1)}


if __name__ == "__main__":
    names = sys.argv[1:] or sorted(WORKLOADS)
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for nm in names:
        data[nm] = run(nm)
        print(nm, data[nm], flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
