"""Writes couette_paper.json: the cylindrical Couette flow of section 3.1.2
run through the FP64 oracle in the paper's own setup, to settle the order of
convergence the paper reports (Fig. 5, "generally second-order").

Setup (section 3.1.2): Re = U1 (R2 - R1)/nu = 10, tau_s = 0.65 and 0.85,
radius ratio R = R1/R2 = 0.5 and 0.8, the MRT rates of section 3, 10
correction iterations.  The outer radius is the unit of length, so the grid
spacing is 1/r2 with r2 the outer radius in lattice units; Re and tau are
held fixed under refinement (diffusive scaling), so the wall speed U1 falls
in proportion to the grid spacing.  f starts at the equilibrium of the
analytic field (Eq. 34 between the rings, rigid rotation inside, rest
outside) and is stepped until the velocity changes by less than STEADY_TOL * U1
over CHUNK steps.

Errors against Eq. 34:
  line_nd   Eq. 35 along theta = pi/2 (the nodes on the ray x = xc, y > yc
            between R1 and R2), in the non-dimensional velocity u / U1;
  line_lu   the same norm in lattice units (u itself);
  ann_rel   relative L2 error over all nodes of the annulus R1 <= r <= R2.
The "readings" family repeats R = 0.5, tau = 0.65 with one alternative
reading of section 2.3 switched on at a time (oracle READINGS), and with the
BGK collision instead of MRT.

Calls only the oracle and the workload geometry.  Run from the repository
root:  python tests/golden/make_couette_paper.py [--cache FILE]
(about 30 min on 8 cores).  With --cache, every finished run is stored in
FILE and reused by a later invocation, so an interrupted run resumes.
"""
import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1803_09380_gb300 import workloads as wl  # noqa: E402

CHUNK = 200
STEADY_TOL = 5e-7
MAIN = [(0.5, 0.65, [10, 20, 40, 80]), (0.5, 0.85, [10, 20, 40, 80]),
        (0.8, 0.65, [20, 40, 80]), (0.8, 0.85, [20, 40, 80])]
READING_LEVELS = [10, 20, 40]
READING_VARIANTS = [("bgk", None), ("interp_moments", {"interp_moments": 1}),
                    ("rho_b_ref", {"rho_b_ref": 1}), ("post_collision", {"post_collision": 1}),
                    ("unit_ds", {"unit_ds": 1})]


def errors(case, ux, uy):
    m = case.meta
    y, x = np.mgrid[0:case.ny, 0:case.nx].astype(np.float64)
    ax, ay = wl.couette_analytic(case, x, y)
    r = np.hypot(x - m["cx"], y - m["cy"])
    ann = (r >= m["r1"]) & (r <= m["r2"])
    rel = math.sqrt(((ux - ax) ** 2 + (uy - ay) ** 2)[ann].sum() / (ax ** 2 + ay ** 2)[ann].sum())
    col = int(round(m["cx"]))
    sel = ann[:, col] & (y[:, col] > m["cy"])
    line = math.sqrt(((ux[sel, col] - ax[sel, col]) ** 2 + (uy[sel, col] - ay[sel, col]) ** 2).mean())
    return {"line_nd": line / m["wall_speed"], "line_lu": line, "ann_rel": rel,
            "line_nodes": int(sel.sum())}


def run(case, reading=None, threaded=True):
    L = oracle.Lattice(case.nx, case.ny, case.tau, n_corr=case.n_corr, mrt=case.mrt,
                       threaded=threaded, reading=reading)
    for b in case.bodies:
        L.add_body(b.xy, b.ds, **b.as_kwargs())
    y, x = np.mgrid[0:case.ny, 0:case.nx].astype(np.float64)
    ax, ay = wl.couette_analytic(case, x, y)
    L.init_equilibrium(1.0, ax, ay)
    u1 = case.meta["wall_speed"]
    prev, steps = None, 0
    while True:
        L.step(CHUNK)
        steps += CHUNK
        _, ux, uy = L.moments()
        if prev is not None:
            d = max(np.abs(ux - prev[0]).max(), np.abs(uy - prev[1]).max())
            if d < STEADY_TOL * u1:
                break
        prev = (ux.copy(), uy.copy())
    rec = {"r2": case.meta["r2"], "n": case.nx, "steps": steps, "u1": u1,
           "markers": case.n_markers, "resid_final_nd": float(L.resid[-1] / u1)}
    rec.update(errors(case, ux, uy))
    return rec


def slopes(runs):
    """Least-squares slope of log error against log grid spacing 1/r2 over
    all levels, and between the two finest levels."""
    h = np.log([1.0 / r["r2"] for r in runs])
    out = {}
    for k in ("line_nd", "line_lu", "ann_rel"):
        e = np.log([r[k] for r in runs])
        out[k] = {"fit": float(np.polyfit(h, e, 1)[0]),
                  "finest_pair": float((e[-1] - e[-2]) / (h[-1] - h[-2]))}
    return out


class Cache:
    """Finished runs keyed by their parameters (optional)."""

    def __init__(self, path):
        self.path = path
        self.runs = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.runs = json.load(f)

    def get(self, key):
        return self.runs.get(key)

    def put(self, key, rec):
        self.runs[key] = rec
        if self.path:
            with open(self.path, "w") as f:
                json.dump(self.runs, f, indent=1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cache", default=None)
    cache = Cache(ap.parse_args().cache)
    threaded = oracle.threaded_available()
    cores = oracle.set_threads(0) if threaded else 1
    doc = {"source": "FP64 oracle, cylindrical Couette flow in the setup of section 3.1.2 "
                     "(Re 10, tau 0.65 / 0.85, R 0.5 / 0.8, MRT rates of section 3, "
                     "10 iterations, diffusive scaling); errors against Eq. 34",
           "steady_tol": STEADY_TOL, "chunk": CHUNK, "threads": cores,
           "note": "slopes are d log(error) / d log(grid spacing): 1 = first order, 2 = second",
           "main": [], "readings": []}
    for ratio, tau, levels in MAIN:
        runs = []
        for r2 in levels:
            key = f"main R{ratio} tau{tau} r{r2}"
            rec = cache.get(key)
            if rec is None:
                t = time.time()
                rec = run(wl.couette_paper(r2, ratio, tau), threaded=threaded)
                rec["seconds"] = round(time.time() - t, 1)
                cache.put(key, rec)
            print(ratio, tau, json.dumps(rec), flush=True)
            runs.append(rec)
        doc["main"].append({"ratio": ratio, "tau": tau, "runs": runs, "slopes": slopes(runs)})
        print(ratio, tau, doc["main"][-1]["slopes"], flush=True)
    for name, reading in READING_VARIANTS:
        runs = []
        for r2 in READING_LEVELS:
            key = f"reading {name} r{r2}"
            rec = cache.get(key)
            if rec is None:
                case = wl.couette_paper(r2, 0.5, 0.65, mrt=(name != "bgk"))
                t = time.time()
                rec = run(case, reading=reading, threaded=threaded)
                rec["seconds"] = round(time.time() - t, 1)
                cache.put(key, rec)
            print(name, json.dumps(rec), flush=True)
            runs.append(rec)
        doc["readings"].append({"reading": name, "ratio": 0.5, "tau": 0.65, "runs": runs,
                                "slopes": slopes(runs)})
        print(name, doc["readings"][-1]["slopes"], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "couette_paper.json"), "w") as f:
        json.dump(doc, f, indent=1)


if __name__ == "__main__":
    main()
