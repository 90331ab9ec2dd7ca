"""Failure paths of the library, each made on the host or through a bounded
device wait -- none faults, traps or hangs the GPU:

  * a device allocator that returns NULL on the k-th call: IBM_ERR_NOMEM,
    the half-built handle is destroyed cleanly and refuses to step, and a
    new lattice afterwards works;
  * markers dense enough to overflow a band node's 32-entry list of covering
    markers: IBM_ERR_BOUNDS (the kernels skip the entries that do not fit);
  * corr_tol below the residual the iterations reach: IBM_WARN_NOT_CONVERGED
    from ibm_step (reported once);
  * finite populations at one node that no collision survives (zero density,
    momentum 2e20): IBM_ERR_DIVERGED from the watchdog scan far from the
    markers, and from the correction kernel's residual check near them;
  * a grid-barrier wait that runs out (one CTA's arrival dropped through the
    test option, 1 ms limit): IBM_ERR_TIMEOUT, and a fresh lattice steps
    normally afterwards."""
import numpy as np
import pytest

from paper_1803_09380_gb300 import ibm
from paper_1803_09380_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _status(fn, *args):
    try:
        fn(*args)
    except ibm.IBMError as e:
        return e.status
    return ibm.IBM_OK


def test_allocation_failure_gives_nomem_and_a_clean_destroy():
    torch = pytest.importorskip("torch")
    case = wl.couette_64()
    calls = {"n": 0, "fail_at": 0, "live": set()}

    def alloc(nbytes, device, stream, ctx):
        calls["n"] += 1
        if calls["n"] == calls["fail_at"]:
            return None
        p = int(torch.cuda.caching_allocator_alloc(int(nbytes), int(device), stream or 0))
        calls["live"].add(p)
        return p

    def release(ptr, device, stream, ctx):
        calls["live"].discard(int(ptr))
        torch.cuda.caching_allocator_delete(int(ptr))

    hooks = (ibm._ALLOC_FN(alloc), ibm._FREE_FN(release))
    ibm.load()
    ibm.ibm_set_allocator(*hooks)
    seen = []
    try:
        # the lattice takes 7 allocations, each body's markers about 25 more
        for k in (1, 4, 7, 9, 20, 33, 40):
            calls["n"], calls["fail_at"] = 0, k
            h = None
            st = ibm.IBM_OK
            try:
                h = ibm.ibm_create_lattice(case.nx, case.ny, case.tau, prec="fp64",
                                           n_corr=case.n_corr)
                for b in case.bodies:
                    ibm.ibm_add_markers(h, b.xy, b.ds, **b.as_kwargs())
            except ibm.IBMError as e:
                st = e.status
            if h is not None and h.value:
                if st != ibm.IBM_OK:
                    assert _status(ibm.ibm_step, h, 1) == ibm.IBM_ERR_INVALID
                ibm.ibm_destroy(h)
            seen.append(st)
            assert not calls["live"], "every device allocation is released by ibm_destroy"
    finally:
        if ibm._torch_hooks is not None:
            ibm.ibm_set_allocator(*ibm._torch_hooks)
        else:
            ibm.ibm_set_allocator(None, None)
    assert seen == [ibm.IBM_ERR_NOMEM] * 7, seen
    with ibm.Lattice.from_case(case, prec="fp64") as lat:
        lat.step(3)
        assert np.all(np.isfinite(lat.moments()[1]))


def test_markers_too_dense_give_bounds():
    """40 markers on one point: every node of their support is covered 40
    times, more than the 32 entries a band node holds."""
    lat = ibm.Lattice(32, 32, 0.8, prec="fp32")
    xy = np.tile([[15.3, 16.2]], (40, 1))
    lat.add_markers(xy, np.ones(40), u=(0.01, 0.0))
    lat.step(1)
    with pytest.raises(ibm.IBMError) as e:
        lat.sync()
    assert e.value.status == ibm.IBM_ERR_BOUNDS and "dense" in str(e.value)
    lat.close()


def test_residual_above_corr_tol_is_reported_by_step():
    case = wl.couette_64()
    with ibm.Lattice.from_case(case, prec="fp64", corr_tol=1e-12) as lat:
        with pytest.raises(ibm.IBMError) as e:
            lat.step(2)
        assert e.value.status == ibm.IBM_WARN_NOT_CONVERGED
        lat.sync()                                   # reported once
        r, st = ibm.ibm_read_fields(lat.h, ibm.FIELD_RESIDUAL, lat.nx, lat.ny, lat.n_corr)
        assert st == ibm.IBM_WARN_NOT_CONVERGED and r[-1] > 1e-12
    with ibm.Lattice.from_case(case, prec="fp64", corr_tol=1.0) as lat:
        lat.step(10)                                 # r^N ~ 1e-5 < 1: no warning
        lat.sync()


def _singular_node(lat, x, y):
    """Finite populations that no collision survives: zero density with a
    momentum of 2e20 (exactly rho = 0 in FP64; in FP32 the velocity squared
    overflows; 16-bit storage cannot hold them and stores Inf)."""
    f = lat.f
    f[:, y, x] = 0.0
    f[1, y, x], f[3, y, x] = 1e20, -1e20
    lat.f = f


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_watchdog_finds_a_diverged_node(prec):
    case = wl.couette_64()
    with ibm.Lattice.from_case(case, prec=prec) as lat:
        lat.step(4)
        _singular_node(lat, 1, 1)                    # far from both rings
        lat.step(1)
        lat.sync()                                   # watchdog off: not seen yet
        ibm.ibm_set_option(lat.h, ibm.IBM_OPT_WATCHDOG_STEPS, 1)
        lat.step(1)
        with pytest.raises(ibm.IBMError) as e:
            lat.sync()
        assert e.value.status == ibm.IBM_ERR_DIVERGED


def test_non_finite_residual_is_diverged():
    case = wl.couette_64()
    with ibm.Lattice.from_case(case, prec="fp64") as lat:
        lat.step(2)
        _singular_node(lat, 42, 32)                  # on the inner ring (radius 10 about 32, 32)
        # the first correction divides by the node's density only in its
        # second-moment pass; the next interpolation reads the NaN
        lat.step(3)
        with pytest.raises(ibm.IBMError) as e:
            lat.sync()
        assert e.value.status == ibm.IBM_ERR_DIVERGED


def test_grid_barrier_wait_runs_out_with_timeout_status():
    """878 markers: the correction kernel runs on 3/4 of the SMs and waits at
    the global-memory grid barrier.  With one CTA's arrival dropped, every
    other CTA's wait ends at the 1 ms limit; the step finishes and the next
    synchronising call returns IBM_ERR_TIMEOUT."""
    case = wl.couette(256)
    lat = ibm.Lattice.from_case(case, prec="fp32")
    lat.step(2)
    lat.sync()
    ibm.ibm_set_option(lat.h, ibm.IBM_OPT_BARRIER_LIMIT_US, 1000)
    ibm.ibm_set_option(lat.h, ibm.IBM_OPT_TEST_DROP_ARRIVAL, 1)
    lat.step(1)
    with pytest.raises(ibm.IBMError) as e:
        lat.sync()
    assert e.value.status == ibm.IBM_ERR_TIMEOUT
    lat.close()
    with ibm.Lattice.from_case(case, prec="fp32") as fresh:
        fresh.step(3)
        fresh.sync()
        assert np.all(np.isfinite(fresh.moments()[1]))
