"""The allocation-free correction entry point (ibm_ib_correct_noalloc) against
the regular path (ibm_step through a handle), called through the C ABI.

This entry point exists for callers that may not call cudaMalloc (code inside
another framework's memory pool, under a fixed device-memory budget, or in a
plug-in limited to the buffers it is given).  It keeps its intermediate
arrays in one fixed device array shared by all calls, so the test makes two
calls in a row on different cases -- and repeats the first -- to show that
what a call leaves behind does not leak into the next.  Every buffer the
entry point reads or writes is allocated here, by the test.

This file is named so that pytest collects it after every other test file."""
import numpy as np
import pytest

from paper_1803_09380_gb300 import ibm
from paper_1803_09380_gb300 import workloads as wl

from _helpers import relerr

pytestmark = pytest.mark.gpu

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.float64)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.float64)


def _case_inputs(case, seed, prec):
    """Initial populations (an equilibrium of seeded random fields, set on a
    handle of the given precision, so that they are representable in it) and
    the flattened marker arrays of every body of the case."""
    h = ibm.Lattice(case.nx, case.ny, case.tau, prec=prec, n_corr=case.n_corr)
    rho, ux, uy = wl.random_fields(case.nx, case.ny, seed, du=0.01, drho=0.005)
    h.init_equilibrium(rho, ux, uy)
    f0 = h.f
    h.close()
    xy = np.concatenate([b.xy for b in case.bodies])
    ds = np.concatenate([b.ds for b in case.bodies])
    uv = []
    for b in case.bodies:
        cx, cy = b.xc
        uv.append(np.stack([b.u[0] - b.omega * (b.xy[:, 1] - cy),
                            b.u[1] + b.omega * (b.xy[:, 0] - cx)], axis=1))
    return f0, xy, ds, np.concatenate(uv)


def _regular_path(case, f0, prec):
    """One ibm_step from f0: the residual history, the summed body force and
    the moments of the corrected state (before the collision)."""
    lat = ibm.Lattice.from_case(case, prec=prec)
    lat.f = f0
    lat.step(1)
    rho, ux, uy = lat.moments()
    out = dict(resid=lat.resid, force=lat.bodies[:, 6:8].sum(axis=0), rho=rho, ux=ux, uy=uy)
    lat.close()
    return out


def _noalloc_path(case, prec, f0, xy, ds, uv):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    ftype = np.float64 if prec == "fp64" else np.float32
    f = torch.from_numpy(np.ascontiguousarray(f0, dtype=ftype)).to(dev)
    dxy = torch.from_numpy(np.ascontiguousarray(xy)).to(dev)
    dds = torch.from_numpy(np.ascontiguousarray(ds)).to(dev)
    duv = torch.from_numpy(np.ascontiguousarray(uv)).to(dev)
    resid = torch.zeros(case.n_corr + 1, dtype=torch.float64, device=dev)
    force = torch.zeros(2, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    ibm.ibm_ib_correct_noalloc(case.nx, case.ny, prec, f.data_ptr(), xy.shape[0], dxy.data_ptr(),
                               dds.data_ptr(), duv.data_ptr(), case.n_corr, resid.data_ptr(),
                               force.data_ptr(), None)
    fc = f.cpu().numpy()
    fd = fc.astype(np.float64)
    rho = fd.sum(axis=0)
    ux = np.tensordot(EX, fd, axes=1) / rho
    uy = np.tensordot(EY, fd, axes=1) / rho
    return dict(resid=resid.cpu().numpy(), force=force.cpu().numpy(), rho=rho, ux=ux, uy=uy), fc


def _compare(a, b, prec):
    if prec == "fp64":
        # the tolerances of the FP64 parity tests
        tol, tol_r = 1e-12, 1e-10
    else:
        # the regular path forms rho and u in float from the same corrected
        # float populations that are summed here in double: rounding of the
        # moments only (~1e-7 of their scale); the residuals and the force
        # come from the same kernels on the same data
        tol, tol_r = 1e-5, 1e-6
    assert relerr(a["rho"], b["rho"]) < tol
    assert relerr(a["ux"], b["ux"]) < tol
    assert relerr(a["uy"], b["uy"]) < tol
    assert relerr(a["resid"], b["resid"]) < tol_r
    assert relerr(a["force"], b["force"]) < tol_r


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_regular_path_on_two_calls_in_a_row(prec):
    first = wl.couette_64()
    second = wl.couette(48, n_corr=7)
    in1 = _case_inputs(first, 5, prec)
    in2 = _case_inputs(second, 6, prec)
    got1, f1 = _noalloc_path(first, prec, *in1)
    got2, _ = _noalloc_path(second, prec, *in2)
    _compare(got1, _regular_path(first, in1[0], prec), prec)
    _compare(got2, _regular_path(second, in2[0], prec), prec)
    again, f1b = _noalloc_path(first, prec, *in1)
    assert np.array_equal(f1, f1b)
    assert np.array_equal(got1["resid"], again["resid"])


def test_noalloc_rejects_sizes_beyond_its_limits():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    buf = torch.zeros(16, dtype=torch.float64, device=dev)
    p = buf.data_ptr()
    with pytest.raises(ibm.IBMError) as e:
        ibm.ibm_ib_correct_noalloc(1024, 1024, "fp64", p, 10, p, p, p, 10)
    assert e.value.status == ibm.IBM_ERR_INVALID and "262144" in str(e.value)
    with pytest.raises(ibm.IBMError) as e:
        ibm.ibm_ib_correct_noalloc(64, 64, "fp64", p, 513, p, p, p, 10)
    assert e.value.status == ibm.IBM_ERR_INVALID and "512" in str(e.value)
