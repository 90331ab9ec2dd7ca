"""Reduced-precision storage: f_i - w_i kept in FP16 or BF16, arithmetic in
FP32, against the FP64 oracle.

Tolerances from the storage rounding: with unit roundoff u16 (2^-11 for
FP16, 2^-8 for BF16) the stored deviations (|f_i - w_i| <= ~4e-3 at wall
speed 0.01) are rounded by ~u16 * 4e-3 per step; the lattice damps these
perturbations, so the steady velocity error stays ~u16 * 4e-3 / |u|max
times a few, i.e. ~1e-3 (FP16) and ~1e-2 (BF16) relative.  The bounds
below are ten times the per-step estimate."""
import math

import numpy as np
import pytest

from paper_1803_09380_gb300 import ibm
from paper_1803_09380_gb300 import workloads as wl

from _helpers import gpu_lattice, oracle_lattice, relerr
from test_couette_convergence import load, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp16": 1e-2, "bf16": 8e-2}


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_f_round_trip_quantises_deviations(prec):
    case = wl.Case("rt", 40, 12, 0.8)
    gpu = gpu_lattice(case, prec)
    rho, ux, uy = wl.random_fields(40, 12, 2, du=0.02, drho=0.01)
    ora = oracle_lattice(case)
    ora.init_equilibrium(rho, ux, uy)
    f0 = ora.f
    gpu.f = f0
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    u16 = 2.0 ** -11 if prec == "fp16" else 2.0 ** -8
    assert np.max(np.abs(gpu.f - f0)) <= u16 * np.max(np.abs(f0 - w)) * 1.01


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_couette_64_velocity_against_oracle(prec):
    """1000 steps of the 64 x 64 Couette case (transient included)."""
    case = wl.couette_64()
    ora = oracle_lattice(case)
    gpu = gpu_lattice(case, prec)
    ora.step(1000)
    gpu.step(1000)
    _, ox, oy = ora.moments()
    _, gx, gy = gpu.moments()
    err = max(relerr(gx, ox), relerr(gy, oy))
    assert err < TOL[prec], err
    assert gpu.resid[-1] < 5 * ora.resid[-1] + 1e-5


@pytest.mark.parametrize("prec,slope_tol", [("fp16", 0.1), ("bf16", 0.3)])
def test_convergence_order_retained(prec, slope_tol):
    """Steady Couette error against Eq. 34 with 16-bit storage at the sweep's
    sizes and step counts (N <= 128): the first-order slope of the FP64
    oracle is kept within slope_tol."""
    runs = [r for r in load()["runs"] if r["n"] <= 128]
    ns, errs = [], []
    for r in runs:
        case = wl.couette(r["n"])
        lat = ibm.Lattice.from_case(case, prec=prec)
        lat.step(r["steps"])
        _, ux, uy = lat.moments()
        errs.append(rel_l2(case, ux, uy))
        ns.append(r["n"])
        lat.close()
    slope = np.polyfit(np.log(ns), np.log(errs), 1)[0]
    print(prec, dict(zip(ns, errs)), "slope", slope)
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert abs(slope - load()["slope_rel_l2_annulus"]) < slope_tol
