"""The 2- and 3-point delta functions (arXiv 1803.09380, Eq. 15a, b) on the
CUDA library against the FP64 oracle."""
import dataclasses
import math

import numpy as np
import pytest

from paper_1803_09380_gb300 import ibm
from paper_1803_09380_gb300 import workloads as wl

from _helpers import field_errors, gpu_lattice, oracle_lattice, relerr

pytestmark = pytest.mark.gpu


def _pair(case, steps, prec="fp64"):
    ora, gpu = oracle_lattice(case), gpu_lattice(case, prec)
    ora.step(steps)
    gpu.step(steps)
    return ora, gpu


@pytest.mark.parametrize("points", [2, 3])
def test_couette_64_fp64(points):
    case = dataclasses.replace(wl.couette_64(), delta_points=points)
    ora, gpu = _pair(case, 60)
    errs = field_errors(gpu, ora)
    assert max(errs["rho"], errs["ux"], errs["uy"], errs["f"]) < 1e-12, errs
    assert errs["fdev"] < 1e-11, errs
    assert relerr(gpu.resid, ora.resid) < 1e-10


@pytest.mark.parametrize("points", [2, 3])
def test_channel_fp64(points):
    case = dataclasses.replace(wl.cylinder(nx=90, ny=41, diameter=10.0, center=(30.0, 20.4), u_in=0.05,
                                           re=20.0, markers=31), delta_points=points)
    ora, gpu = _pair(case, 50)
    errs = field_errors(gpu, ora)
    assert max(errs["rho"], errs["ux"], errs["uy"], errs["f"]) < 1e-12, errs


@pytest.mark.parametrize("points", [2, 3])
def test_settling_disk_fp64(points):
    """Moving markers are re-weighted every step with the chosen kernel."""
    case = dataclasses.replace(wl.settling_single(nx=60, ny=120, diameter=10.0, density_ratio=1.3,
                                                  gravity=2e-4), delta_points=points)
    ora, gpu = _pair(case, 50)
    errs = field_errors(gpu, ora)
    assert errs["rho"] < 1e-12 and errs["f"] < 1e-12, errs
    assert max(errs["ux"], errs["uy"]) < 1e-10, errs
    assert relerr(gpu.bodies[:, 2:4], ora.bodies[:, 2:4]) < 1e-10


def test_three_point_line_halves_the_residual():
    """The closed form the oracle is pinned to, reproduced on the GPU: a
    straight periodic line under the 3-point kernel contracts by 1/2."""
    n = 32
    xy = np.stack([np.arange(n) + 0.37, np.full(n, 11.3)], axis=1)
    lat = ibm.Lattice(n, n, 0.8, prec="fp64", n_corr=8, delta_points=3)
    U = (0.01, -0.006)
    lat.add_markers(xy, np.ones(n), u=U, xc=(0.0, 11.3))
    lat.step(1)
    mag = math.hypot(*U)
    r = lat.resid
    for k in range(9):
        assert abs(r[k] - mag * 0.5 ** k) < 1e-15 + 1e-12 * mag


def test_invalid_kernel_is_rejected():
    with pytest.raises(ibm.IBMError):
        ibm.Lattice(16, 16, 0.8, prec="fp64", delta_points=5)
