"""Shared helpers of the parity tests: build the same case on the oracle and
on the CUDA library, and compare normwise."""
import numpy as np

import oracle
from paper_1803_09380_gb300 import ibm

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def oracle_lattice(case, n_corr=None):
    L = oracle.Lattice(case.nx, case.ny, case.tau, case.rho0, case.bc, case.wall_u,
                       case.inlet_u, case.n_corr if n_corr is None else n_corr, mrt=case.mrt,
                       delta_points=case.delta_points)
    for b in case.bodies:
        L.add_body(b.xy, b.ds, **b.as_kwargs())
    return L


def gpu_lattice(case, prec, n_corr=None):
    lat = ibm.Lattice(case.nx, case.ny, case.tau, case.rho0, prec, case.bc, case.wall_u,
                      case.inlet_u, case.n_corr if n_corr is None else n_corr, mrt=case.mrt,
                      delta_points=case.delta_points)
    for b in case.bodies:
        lat.add_markers(b.xy, b.ds, **b.as_kwargs())
    return lat


def relerr(a, b):
    """||a - b||_inf / ||b||_inf (absolute when b is identically zero)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.max(np.abs(a - b)) if a.size else 0.0
    s = np.max(np.abs(b)) if b.size else 0.0
    return d / s if s > 0 else d


def field_errors(gpu, ora, rho0=1.0):
    """Normwise relative errors: rho, u_x, u_y of the last corrected state,
    the density deviation rho - rho0, the post-stream populations f, and
    their deviations f - w_i rho0; plus the largest absolute density
    difference (drho_abs) and the scale of rho - rho0 (drho_scale).

    Both sides form rho as a nine-term sum of populations ~w_i, so each
    carries a rounding of a few ulp of rho0 whatever the size of rho - rho0;
    the density deviation is therefore held to an absolute floor of a few
    ulp as well as to the relative tolerance (see density_ok).  The deviation
    error f - w_i is reported separately for the same reason."""
    gr, gx, gy = gpu.moments()
    orr, ox, oy = ora.moments()
    fg, fo = gpu.f, ora.f
    w = W[:, None, None] * rho0
    return {
        "rho": relerr(gr, orr),
        "drho": relerr(gr - rho0, orr - rho0),
        "drho_abs": float(np.max(np.abs(gr - orr))),
        "drho_scale": float(np.max(np.abs(orr - rho0))),
        "ux": relerr(gx, ox),
        "uy": relerr(gy, oy),
        "f": relerr(fg, fo),
        "fdev": relerr(fg - w, fo - w),
    }


def density_ok(errs, tol, rho0=1.0, ulps=16, eps=2.0 ** -53):
    """rho - rho0 within tol of its own scale, or within `ulps` units in the
    last place of rho0 (the rounding floor of a nine-term sum ~rho0)."""
    return errs["drho_abs"] <= tol * errs["drho_scale"] + ulps * eps * rho0
