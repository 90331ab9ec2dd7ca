"""The serving layer: many independent cases resident at once, admitted as
memory and slots free up, results identical alone and in the mix."""
import numpy as np
import pytest

from paper_1803_09380_gb300 import ibm
from paper_1803_09380_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FIELDS = (ibm.FIELD_RHO, ibm.FIELD_UX, ibm.FIELD_UY, ibm.FIELD_BODIES, ibm.FIELD_RESIDUAL)


def _mix():
    stream = wl.serving_stream(n_requests=14, seed=7, steps=150, couette_n=(40, 160), cyl_ny=(40, 90),
                               box=(80, 200), disk_d=(10.0, 16.0))
    return [(c, s) for _, c, s in stream]


def _run(cases, max_active, prec="fp32", steps_per_launch=40):
    with ibm.Server(max_active=max_active, steps_per_launch=steps_per_launch) as srv:
        ids = [srv.submit(c, s, prec=prec) for c, s in cases]
        srv.wait()
        st = srv.stats()
        res = [{f: srv.result(i, f) for f in FIELDS} for i in ids]
    return res, st


def test_results_are_the_same_alone_and_in_the_mix():
    cases = _mix()
    mixed, st = _run(cases, max_active=8)
    assert st["completed"] == len(cases) and st["failed"] == 0
    for (c, s), got in zip(cases, mixed):
        alone, _ = _run([(c, s)], max_active=1)
        for f in FIELDS:
            assert np.array_equal(alone[0][f], got[f]), (c.name, f)


def test_server_matches_a_plain_handle():
    case = wl.couette(96)
    (res,), _ = _run([(case, 120)], max_active=1, prec="fp64")
    lat = ibm.Lattice.from_case(case, prec="fp64")
    lat.step(120)
    rho, ux, uy = lat.moments()
    assert np.array_equal(res[ibm.FIELD_UX], ux) and np.array_equal(res[ibm.FIELD_RHO], rho)
    assert np.array_equal(res[ibm.FIELD_RESIDUAL], lat.resid)


def test_admission_respects_the_memory_budget():
    cases = [(wl.couette(128), 60) for _ in range(6)]
    with ibm.Server(max_active=6, steps_per_launch=20, max_device_bytes=1.0) as srv:
        for c, s in cases:
            srv.submit(c, s)
        peak = 0
        while True:
            srv.progress()
            st = srv.stats()
            peak = max(peak, st["active"])
            if st["completed"] + st["failed"] == len(cases):
                break
        assert peak == 1                      # a budget below one case admits one at a time
        assert st["completed"] == len(cases)


def test_latency_percentiles_are_ordered():
    _, st = _run(_mix()[:8], max_active=4)
    assert 0 < st["p50_ms"] <= st["p95_ms"] <= st["p99_ms"]
    assert st["solves_per_s"] > 0 and st["mlups"] > 0


def test_failed_case_reports_its_error():
    bad = wl.Case("bad", 32, 32, 0.8, bc=(1, 1, 1, 1),
                  bodies=[wl.Body(np.array([[0.5, 16.0]]), np.array([1.0]))])
    with ibm.Server(max_active=2) as srv:
        i = srv.submit(bad, 10)
        j = srv.submit(wl.couette(48), 10)
        srv.wait()
        with pytest.raises(ibm.IBMError) as e:
            srv.result(i, ibm.FIELD_UX)
        assert e.value.status == ibm.IBM_ERR_INVALID
        assert srv.result(j, ibm.FIELD_UX).shape == (48, 48)
