"""Error of the reduced precisions against FP64, per workload configuration.

Cylinder: the 1600 x 800 channel (D = 40, 126 markers, centre (400, 400),
uniform equilibrium inflow U = 0.05 at -x, zero-gradient outlet, free-slip
walls, BGK, Re 20).  Against the FP64 oracle after 100 steps (velocity field),
and against the library's FP64 mode -- itself equal to the oracle at 1e-12 --
after 20,000 steps (drag coefficient and velocity field; the oracle would
need hours for that).  Measured on GB300 after 100,000 steps: FP32 C_d within
0.08 % (Re 20) and 0.11 % (Re 40) of FP64, velocity within 1e-3; FP16
deviation storage 6 % and 11 % on C_d; BF16 43 % and 48 % (its 8-bit
mantissa cannot hold the deviations f - w_i of this flow).

Settling disks (drafting-kissing-tumbling pair, two disks D = 20 in a 200 x
800 bounce-back box, density ratio 1.01): against the FP64 oracle after
5,000 steps (body positions, velocities, velocity field).  Measured after
50,000 steps against the FP64 library: FP32 positions within 0.02 lattice
units, FP16 0.84, BF16 1.65."""
import numpy as np
import pytest

import oracle
from paper_1803_09380_gb300 import ibm
from paper_1803_09380_gb300 import workloads as wl

from _helpers import gpu_lattice, relerr

pytestmark = pytest.mark.gpu


def _cylinder(re=20.0):
    return wl.cylinder(nx=1600, ny=800, diameter=40.0, center=(400.0, 400.0), u_in=0.05, re=re,
                       markers=126)


def test_cylinder_channel_against_the_oracle_after_100_steps():
    case = _cylinder()
    ora = oracle.Lattice(case.nx, case.ny, case.tau, bc=case.bc, wall_u=case.wall_u,
                         inlet_u=case.inlet_u, n_corr=case.n_corr, threaded=oracle.threaded_available())
    for b in case.bodies:
        ora.add_body(b.xy, b.ds, **b.as_kwargs())
    ora.step(100)
    _, ox, oy = ora.moments()
    bound = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 1e-2, "bf16": 1e-1}
    for prec, tol in bound.items():
        g = gpu_lattice(case, prec, None)
        g.step(100)
        _, gx, gy = g.moments()
        g.close()
        assert relerr(gx, ox) < tol and relerr(gy, oy) < max(tol, 1e-12), (prec, relerr(gx, ox))


def test_cylinder_channel_drag_per_precision_after_20000_steps():
    case = _cylinder()
    q = 0.5 * case.rho0 * case.inlet_u[0] ** 2 * case.meta["diameter"]
    out = {}
    for prec in ("fp64", "fp32", "fp16", "bf16"):
        g = gpu_lattice(case, prec, None)
        cd = []
        for _ in range(20):
            g.step(1000, flags=ibm.STEP_NO_MACRO)
            cd.append(g.bodies[0][6] / q)
        g.step(1)
        out[prec] = (np.mean(cd[-5:]), g.moments()[1])
        g.close()
    cd64, u64 = out["fp64"]
    assert 1.0 < cd64 < 2.5
    # FP32: the same drag to 0.5 %, the same field to 5e-3 of its largest value
    assert abs(out["fp32"][0] / cd64 - 1) < 5e-3 and relerr(out["fp32"][1], u64) < 5e-3
    # 16-bit deviation storage: FP16 within 15 % on the drag; BF16 is stated,
    # not held to a bound (tens of per cent: its mantissa is too short here)
    assert abs(out["fp16"][0] / cd64 - 1) < 0.15
    assert np.isfinite(out["bf16"][0])


def test_settling_pair_against_the_oracle_after_5000_steps():
    case = wl.settling_pair()
    ora = oracle.Lattice(case.nx, case.ny, case.tau, bc=case.bc, n_corr=case.n_corr,
                         threaded=oracle.threaded_available())
    for b in case.bodies:
        ora.add_body(b.xy, b.ds, **b.as_kwargs())
    ora.step(5000)
    bo = ora.bodies
    bound = {"fp64": (1e-9, 1e-9), "fp32": (1e-3, 1e-3), "fp16": (0.1, 0.1), "bf16": (0.2, 0.2)}
    for prec, (tp, tv) in bound.items():
        g = gpu_lattice(case, prec, None)
        g.step(5000)
        bg = g.bodies
        g.close()
        assert np.max(np.abs(bg[:, 0:2] - bo[:, 0:2])) < tp, prec
        assert relerr(bg[:, 2:4], bo[:, 2:4]) < tv, prec
