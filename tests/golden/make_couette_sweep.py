"""Writes couette_sweep.json: steady-state error of the FP64 oracle against the
analytic cylindrical Couette profile (Eq. 34, section 3.1.2) on N x N
lattices with radii 0.156 N and 0.39 N, inner wall speed 0.01, tau = 0.8,
10 correction iterations.  Calls only the oracle and the workload geometry.

Run from the repository root:  python tests/golden/make_couette_sweep.py
"""
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

SIZES = [32, 48, 64, 96, 128, 192]
CHUNK = 500
TOL = 1e-9          # steady when max |u(t) - u(t - CHUNK)| < TOL * max |u|


def errors(case, ux, uy):
    """Relative L2 error over the annulus r1 <= r <= r2, and the absolute
    L2 error of Eq. 35 along the profile theta = pi/2 (x = centre)."""
    m = case.meta
    y, x = np.mgrid[0:case.ny, 0:case.nx].astype(np.float64)
    ax, ay = wl.couette_analytic(case, x, y)
    r = np.hypot(x - m["cx"], y - m["cy"])
    ann = (r >= m["r1"]) & (r <= m["r2"])
    rel = math.sqrt(((ux - ax) ** 2 + (uy - ay) ** 2)[ann].sum() / (ax ** 2 + ay ** 2)[ann].sum())
    col = int(round(m["cx"]))
    sel = ann[:, col] & (y[:, col] > m["cy"])
    prof = math.sqrt(((ux[sel, col] - ax[sel, col]) ** 2 + (uy[sel, col] - ay[sel, col]) ** 2).mean())
    return rel, prof


def run(n):
    case = wl.couette(n)
    L = oracle.Lattice(case.nx, case.ny, case.tau, n_corr=case.n_corr)
    for b in case.bodies:
        L.add_body(b.xy, b.ds, **b.as_kwargs())
    prev = None
    steps = 0
    while True:
        L.step(CHUNK)
        steps += CHUNK
        _, ux, uy = L.moments()
        if prev is not None:
            d = max(np.abs(ux - prev[0]).max(), np.abs(uy - prev[1]).max())
            if d < TOL * max(np.abs(ux).max(), np.abs(uy).max()):
                break
        prev = (ux.copy(), uy.copy())
    rel, prof = errors(case, ux, uy)
    return {"n": n, "steps": steps, "rel_l2_annulus": rel, "l2_profile": prof,
            "resid_final": float(L.resid[-1]), "markers": case.n_markers}


def main():
    out = []
    for n in SIZES:
        t = time.time()
        rec = run(n)
        rec["seconds"] = round(time.time() - t, 1)
        print(json.dumps(rec), flush=True)
        out.append(rec)
    ln = np.log([r["n"] for r in out])
    slope_rel = float(np.polyfit(ln, np.log([r["rel_l2_annulus"] for r in out]), 1)[0])
    slope_prof = float(np.polyfit(ln, np.log([r["l2_profile"] for r in out]), 1)[0])
    doc = {"source": "FP64 oracle, cylindrical Couette flow (section 3.1.2, Eqs. 32-35), "
                     "radii 0.156 N / 0.39 N, wall speed 0.01, tau 0.8, 10 iterations",
           "steady_tol": TOL, "runs": out,
           "slope_rel_l2_annulus": slope_rel, "slope_l2_profile": slope_prof}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "couette_sweep.json"), "w") as f:
        json.dump(doc, f, indent=1)
    print("slopes", slope_rel, slope_prof)


if __name__ == "__main__":
    main()
