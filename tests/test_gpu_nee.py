"""Non-equilibrium-extrapolation inlet and outlet (the boundary scheme of
the cylinder channel in section 3.2) on the CUDA library against the FP64
oracle.  The boundary columns' own post-stream populations that would come
from outside are never read by either side (each step rebuilds the column),
so f is compared on the other columns; the moments everywhere."""
import dataclasses

import numpy as np
import pytest

from paper_1803_09380_gb300 import ibm
from paper_1803_09380_gb300 import workloads as wl

from _helpers import gpu_lattice, oracle_lattice, relerr

pytestmark = pytest.mark.gpu
NEE = (wl.INLET_NEE, wl.OUTLET_NEE)


def _uniform(case, u):
    shp = (case.ny, case.nx)

    def init(ora, gpu):
        for lat in (ora, gpu):
            lat.init_equilibrium(np.ones(shp), np.full(shp, u), np.zeros(shp))
    return init


def _pair(case, steps, prec="fp64", init=None):
    ora, gpu = oracle_lattice(case), gpu_lattice(case, prec)
    if init is not None:
        init(ora, gpu)
    ora.step(steps)
    gpu.step(steps)
    return ora, gpu


def _errors(gpu, ora):
    gr, gx, gy = gpu.moments()
    orr, ox, oy = ora.moments()
    scale = max(np.abs(ox).max(), np.abs(oy).max())
    return {"rho": relerr(gr, orr),
            "u": max(np.abs(gx - ox).max(), np.abs(gy - oy).max()) / scale,
            "f": relerr(gpu.f[:, :, 1:-1], ora.f[:, :, 1:-1])}


def _cylinder_channel(nx=90, ny=41, **kw):
    case = wl.cylinder(nx=nx, ny=ny, diameter=10.0, center=(30.0, ny / 2.0 - 0.1), u_in=0.05, re=20.0,
                       markers=31)
    return dataclasses.replace(case, bc=NEE + (wl.FREESLIP, wl.FREESLIP), **kw)


def test_cylinder_channel_fp64():
    case = _cylinder_channel()
    ora, gpu = _pair(case, 80, init=_uniform(case, 0.05))
    errs = _errors(gpu, ora)
    assert max(errs.values()) < 1e-12, errs
    assert relerr(gpu.bodies[:, 6:9], ora.bodies[:, 6:9]) < 1e-10


def test_channel_between_walls_fp64_both_step_kinds():
    for steps in (1, 2, 61):
        case = wl.Case("poiseuille", 60, 15, 0.8, bc=NEE + (wl.BOUNCEBACK, wl.BOUNCEBACK), inlet_u=(0.02, 0.0))
        ora, gpu = _pair(case, steps, init=_uniform(case, 0.02))
        errs = _errors(gpu, ora)
        assert max(errs.values()) < 1e-12, (steps, errs)


def test_mrt_channel_fp64():
    case = _cylinder_channel(mrt=ibm.PAPER_MRT_RATES)
    ora, gpu = _pair(case, 60, init=_uniform(case, 0.05))
    errs = _errors(gpu, ora)
    assert max(errs.values()) < 1e-12, errs


def test_wide_channel_fp32():
    """Full vector spans between the extrapolation columns, FP32 against the
    FP64 oracle (velocity relative to the flow speed)."""
    case = _cylinder_channel(nx=1030, ny=40)
    ora, gpu = _pair(case, 40, prec="fp32", init=_uniform(case, 0.05))
    errs = _errors(gpu, ora)
    assert errs["u"] < 1e-4 and errs["f"] < 1e-6, errs


def test_uniform_stream_is_kept():
    case = wl.Case("stream", 70, 9, 0.7, bc=NEE + (wl.PERIODIC, wl.PERIODIC), inlet_u=(0.05, 0.0))
    gpu = gpu_lattice(case, "fp64")
    shp = (case.ny, case.nx)
    gpu.init_equilibrium(np.ones(shp), np.full(shp, 0.05), np.zeros(shp))
    gpu.step(120)
    rho, ux, uy = gpu.moments()
    assert np.abs(rho - 1).max() < 1e-13 and np.abs(ux - 0.05).max() < 1e-13 and np.abs(uy).max() < 1e-13


def test_markers_next_to_an_extrapolation_side_are_rejected():
    lat = ibm.Lattice(40, 20, 0.8, prec="fp64", bc=NEE + (wl.FREESLIP, wl.FREESLIP), inlet_u=(0.05, 0.0))
    with pytest.raises(ibm.IBMError):
        lat.add_markers(np.array([[2.5, 10.0]]), np.array([1.0]))
    with pytest.raises(ibm.IBMError):
        ibm.Lattice(40, 20, 0.8, prec="fp64", bc=(wl.OUTLET_NEE, wl.INLET_NEE, 2, 2))
