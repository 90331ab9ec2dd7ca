"""Steady cylindrical Couette flow (section 3.1.2, Eq. 34) on a 128 x 128
lattice -- radii 0.156 N and 0.39 N, inner wall speed 0.01, tau = 0.8, 10
correction iterations -- after 20,500 steps, the step count at which the
oracle's grid-refinement sweep found the 128^2 field steady (velocity change
below 1e-9 of its maximum over 500 steps).

FP32 storage and arithmetic against the FP64 oracle, element by element:
u_x and u_y within 1e-4 of the field's largest value at every node (the
FP32 bound for steady velocity).  The FP64 library over the same 20,500
steps stays at the FP64 bound.  The oracle runs once, on all host cores (its
threaded build is bitwise the serial one)."""
import numpy as np
import pytest

import oracle
from paper_1803_09380_gb300 import workloads as wl

from _helpers import field_errors, gpu_lattice, relerr

pytestmark = pytest.mark.gpu

STEPS = 20500


@pytest.fixture(scope="module")
def steady():
    case = wl.couette(128)
    ora = oracle.Lattice(case.nx, case.ny, case.tau, n_corr=case.n_corr,
                         threaded=oracle.threaded_available())
    for b in case.bodies:
        ora.add_body(b.xy, b.ds, **b.as_kwargs())
    ora.step(STEPS)
    return case, ora


def test_fp32_steady_velocity_element_by_element(steady):
    case, ora = steady
    gpu = gpu_lattice(case, "fp32", None)
    gpu.step(STEPS)
    _, gx, gy = gpu.moments()
    orho, ox, oy = ora.moments()
    scale = max(np.abs(ox).max(), np.abs(oy).max())
    ex = np.abs(gx - ox) / scale
    ey = np.abs(gy - oy) / scale
    assert ex.max() < 1e-4 and ey.max() < 1e-4, (ex.max(), ey.max())
    # nodes where the flow is fast enough for a pointwise relative error:
    # the annulus and the rigidly turning interior
    mag = np.hypot(ox, oy)
    fast = mag > 0.1 * mag.max()
    assert np.max(np.hypot(gx - ox, gy - oy)[fast] / mag[fast]) < 1e-3
    errs = field_errors(gpu, ora)
    # FP32 keeps rho ~ 1 to ~6e-8 a step; 20,500 steps of rounding leave
    # ~1e-6 (measured 9.4e-7), against a rho - rho0 scale of 2.4e-4
    assert errs["drho_abs"] < 4e-6, errs
    gpu.close()


def test_fp64_after_the_steady_run_stays_at_the_fp64_bound(steady):
    case, ora = steady
    gpu = gpu_lattice(case, "fp64", None)
    gpu.step(STEPS)
    errs = field_errors(gpu, ora)
    assert max(errs["rho"], errs["ux"], errs["uy"], errs["f"]) < 1e-12, errs
    assert relerr(gpu.resid, ora.resid) < 1e-10
    gpu.close()
