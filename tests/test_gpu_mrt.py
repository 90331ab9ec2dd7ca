"""MRT collision (arXiv 1803.09380, Eqs. 2, 5, 6; rates of section 3) on the
CUDA library against the FP64 oracle, and the correction kernel's results
independent of its CTA count."""
import dataclasses

import numpy as np
import pytest

from paper_1803_09380_gb300 import ibm
from paper_1803_09380_gb300 import workloads as wl

from _helpers import density_ok, field_errors, gpu_lattice, oracle_lattice, relerr

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL_MOVING = 1e-10
PAPER = ibm.PAPER_MRT_RATES


def _mrt(case, rates=PAPER):
    return dataclasses.replace(case, mrt=tuple(rates))


def _pair(case, steps, prec="fp64", init=None):
    ora, gpu = oracle_lattice(case), gpu_lattice(case, prec)
    if init is not None:
        init(ora, gpu)
    ora.step(steps)
    gpu.step(steps)
    return ora, gpu


def _random_init(seed):
    def init(ora, gpu):
        ora.init_equilibrium(*wl.random_fields(ora.nx, ora.ny, seed))
        f0 = ora.f + wl.random_perturbation(ora.nx, ora.ny, seed + 1, 1e-4)
        ora.f = f0
        gpu.f = f0
    return init


def _check(gpu, ora, tol, tol_dev=None):
    errs = field_errors(gpu, ora)
    lim = {"fdev": 10 * tol if tol_dev is None else tol_dev}
    for k in ("rho", "ux", "uy", "f", "fdev"):
        assert errs[k] < lim.get(k, tol), (k, errs)
    assert density_ok(errs, tol), ("rho - rho0", errs)


@pytest.mark.parametrize("steps", [1, 2, 51])
def test_mrt_periodic_random_state_fp64(steps):
    """Random non-equilibrium state (every moment off equilibrium), 70 x 45
    periodic: both AA step kinds with the MRT operator."""
    ora, gpu = _pair(_mrt(wl.Case("p", 70, 45, 0.73)), steps, init=_random_init(5))
    _check(gpu, ora, TOL64)


def test_mrt_couette_64_fp64_100_steps():
    ora, gpu = _pair(_mrt(wl.couette_64()), 100)
    _check(gpu, ora, TOL64)
    assert relerr(gpu.resid, ora.resid) < 1e-10


def test_mrt_channel_fp64():
    case = _mrt(wl.cylinder(nx=90, ny=41, diameter=10.0, center=(30.0, 20.4), u_in=0.05, re=20.0,
                            markers=31))
    ora, gpu = _pair(case, 80)
    _check(gpu, ora, TOL64)


def test_mrt_box_walls_and_settling_disk_fp64():
    wall_u = np.zeros(8)
    wall_u[6] = 0.02
    case = wl.settling_single(nx=60, ny=120, diameter=10.0, density_ratio=1.3, gravity=2e-4)
    case = _mrt(dataclasses.replace(case, wall_u=tuple(wall_u)), rates=(1.4, 1.0, 1.2))
    ora, gpu = _pair(case, 60)
    errs = field_errors(gpu, ora)
    assert errs["rho"] < TOL64 and errs["f"] < TOL64, errs
    assert max(errs["ux"], errs["uy"], errs["fdev"]) < TOL_MOVING, errs
    assert relerr(gpu.bodies[:, 2:4], ora.bodies[:, 2:4]) < 1e-10


def test_mrt_wide_fp32():
    """FP32 vector spans and band segments with MRT against the FP64 oracle."""
    ora, gpu = _pair(_mrt(wl.couette(300)), 60, prec="fp32")
    errs = field_errors(gpu, ora)
    assert errs["ux"] < 1e-4 and errs["uy"] < 1e-4 and errs["f"] < 1e-6, errs


@pytest.mark.parametrize("prec,tol", [("fp16", 1e-2), ("bf16", 8e-2)])
def test_mrt_16bit_storage(prec, tol):
    ora, gpu = _pair(_mrt(wl.couette_64()), 300, prec=prec)
    _, ox, oy = ora.moments()
    _, gx, gy = gpu.moments()
    assert relerr(gx, ox) < tol and relerr(gy, oy) < tol


def test_mrt_with_equal_rates_matches_bgk():
    """Every rate 1/tau: the MRT kernels agree with the BGK kernels to
    rounding (the two are algebraically identical)."""
    case = wl.couette(80)
    w = 1.0 / case.tau
    a = gpu_lattice(case, "fp64")
    b = gpu_lattice(_mrt(case, rates=(w, w, w)), "fp64")
    a.step(40)
    b.step(40)
    assert relerr(b.f, a.f) < 1e-14
    assert relerr(b.moments()[1], a.moments()[1]) < 1e-11


def test_mrt_rates_are_validated():
    with pytest.raises(ibm.IBMError):
        ibm.Lattice(16, 16, 0.8, prec="fp64", mrt=(2.5, 1.0, 1.0))
    lat = ibm.Lattice(16, 16, 0.8, prec="fp64", mrt=(0.0, 0.0, 0.0))   # 0: section 3 values
    lat.step(2)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_correction_results_do_not_depend_on_cta_count(prec):
    """The correction kernel's sums use fixed chunks and trees, so any CTA
    count (one CTA with a block barrier, or a grid barrier over many) and
    any CTA size give bitwise the same state, residuals and body forces."""
    case = wl.couette(256)
    ref = None
    for ctas, threads in ((0, 256), (1, 256), (3, 256), (152, 256), (2, 512), (19, 1024)):
        lat = gpu_lattice(case, prec)
        lat.set_ib_ctas(ctas)
        lat.set_ib_threads(threads)
        lat.step(12)
        got = (lat.f, lat.resid, lat.bodies)
        if ref is None:
            ref = got
        else:
            for g, r in zip(got, ref):
                assert np.array_equal(g, r), ctas


def test_autotuned_correction_grid_keeps_the_trajectory():
    """The autotuner's candidate runs are ordinary steps: after it, the
    lattice is where the same number of steps with any fixed setting puts
    it, bit for bit; it returns one of the candidates and a positive time."""
    case = wl.couette(256)
    tuned = gpu_lattice(case, "fp32")
    cand = [1, 4, 16, 57, 76, 152]
    best, us = tuned.autotune_ib(cand, steps_each=5)
    assert best in cand and us > 0
    ref = gpu_lattice(case, "fp32")
    ref.step(len(cand) * (2 + 5))
    tuned.step(3)
    ref.step(3)
    assert np.array_equal(tuned.f, ref.f) and np.array_equal(tuned.resid, ref.resid)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_changing_the_correction_grid_on_a_live_lattice(prec):
    """Grid sizes that are not multiples of each other, switched between
    steps of one lattice (the grid barrier's counter restarts for each new
    size): no barrier runs out and the trajectory is bitwise that of a
    fixed setting."""
    case = wl.couette(256)
    live = gpu_lattice(case, prec)
    for ctas in (76, 95, 152, 57, 114):
        live.set_ib_ctas(ctas)
        live.step(3)
    ref = gpu_lattice(case, prec)
    ref.step(15)
    assert np.array_equal(live.f, ref.f) and np.array_equal(live.resid, ref.resid)
    assert np.array_equal(live.bodies, ref.bodies)
