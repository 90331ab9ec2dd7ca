"""Writes tgv_sweep.json: the oracle's L2 velocity error (Eq. 31) against
Eq. 30 at t* = 1 for the Taylor-Green vortices with an artificial cylinder
(section 3.1.1), L = 10, 20, 40, FP64.  Calls only the oracle.

Protocol: f starts at the equilibrium of Eq. 30 at t = 0; before step k
(k = 0 .. T) the markers get the velocity of Eq. 30 at t = k; after T + 1
steps the moments of the corrected state are those of time T, compared
with Eq. 30 at t = T over all nodes."""
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))

import oracle  # noqa: E402
from paper_1803_09380_gb300 import workloads as wl  # noqa: E402


def run(L):
    case = wl.taylor_green(L)
    lat = oracle.Lattice(case.nx, case.ny, case.tau, n_corr=case.n_corr)
    b = case.bodies[0]
    lat.add_body(b.xy, b.ds, **b.as_kwargs())
    yy, xx = np.mgrid[0:case.ny, 0:case.nx].astype(np.float64)
    lat.init_equilibrium(*wl.taylor_green_fields(case, xx, yy, 0.0))
    T = wl.taylor_green_steps(case)
    for k in range(T + 1):
        _, ux, uy = wl.taylor_green_fields(case, b.xy[:, 0], b.xy[:, 1], float(k))
        lat.set_marker_velocities(np.stack([ux, uy], axis=1))
        lat.step(1)
    _, gx, gy = lat.moments()
    _, ax, ay = wl.taylor_green_fields(case, xx, yy, float(T))
    return math.sqrt(np.mean((gx - ax) ** 2 + (gy - ay) ** 2)), T


def main():
    out = {"case": "Taylor-Green vortices with a cylinder of diameter L, Re 10, tau 0.65, t* = 1",
           "norm": "Eq. 31 over all nodes", "L": [], "l2": [], "steps": []}
    for L in (10, 20, 40):
        t0 = time.time()
        e, T = run(L)
        out["L"].append(L)
        out["l2"].append(e)
        out["steps"].append(T)
        print(L, T, e, round(time.time() - t0, 1), flush=True)
    ls, es = np.log(out["L"]), np.log(out["l2"])
    out["slope"] = float(np.polyfit(ls, es, 1)[0])
    with open(os.path.join(HERE, "tgv_sweep.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("slope", out["slope"])


if __name__ == "__main__":
    main()
