"""Run the FP64 oracle on a full-size benchmark workload and store its results.

    python -m oracle.record_reference spheres128 uzawa    # -> tests/golden/oracle_spheres128_uzawa.json

The stored file holds the oracle's permeability, outer / inner iteration counts and
per-phase timings for one preconditioner.  The GPU parity tests compare the CUDA path
with it at full size, and the CPU baseline of bench.py uses its iteration counts to
scale a bounded timing sample to whole solves.  Everything in the file comes from this
script and the oracle package only.
"""

from __future__ import annotations

import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

from oracle import krylov, stokes  # noqa: E402
from paper_2307_05266_gb300 import synth  # noqa: E402

WORKLOADS = {
    # 128^3 periodic overlapping spheres, radii U[4, 8), porosity 0.40, seed 0, f = e_x
    "spheres128": dict(make=lambda: synth.sphere_packing(128, 4.0, 8.0, 0.40, 0),
                       force=(1.0, 0.0, 0.0), tol=1e-8),
    # a 64^3 version of the same recipe (quick full-path comparison)
    "spheres64": dict(make=lambda: synth.sphere_packing(64, 4.0, 8.0, 0.40, 0),
                      force=(1.0, 0.0, 0.0), tol=1e-8),
}
PRECONDS = {"uzawa": stokes.UZAWA, "simple": stokes.SIMPLE}


def run(workload: str, precond: str) -> dict:
    w = WORKLOADS[workload]
    mask = w["make"]()
    t0 = time.perf_counter()
    prob = stokes.StokesProblem(mask)
    t_asm = time.perf_counter() - t0
    opts = stokes.Options(precond=PRECONDS[precond], tol=w["tol"])
    t0 = time.perf_counter()
    out, g = prob.solve(w["force"], opts)
    t_solve = time.perf_counter() - t0
    t0 = time.perf_counter()
    rec = prob.recover_velocity(w["force"], out.p, opts)
    t_rec = time.perf_counter() - t0
    k = [prob.permeability(rec.x, a) for a in range(prob.geo.d)]
    return {
        "workload": workload, "precond": precond,
        "n_unknown": int(prob.geo.n_u), "n_fluid": int(prob.geo.n_p),
        "n_components": int(prob.n_comp),
        "k": k, "outer_iters": out.outer_iters, "status": out.status,
        "rel_res": out.rel_res, "inner_iters_A": out.inner_iters_A,
        "inner_iters_S": out.inner_iters_S, "recovery_iters": rec.iters,
        "g_norm": float(np.linalg.norm(g)),
        "seconds": {"assemble": t_asm, "solve": t_solve, "recover": t_rec},
        "host": platform.machine(), "numpy": np.__version__,
        "ok": out.status == krylov.OK,
    }


if __name__ == "__main__":
    wl, pc = sys.argv[1], sys.argv[2]
    res = run(wl, pc)
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{wl}_{pc}.json")
    with open(path, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res))
