"""The batched serving mode: one persistent kernel per round of steps takes
every resident case's correction tasks and collide+stream tiles from one
work queue.  Each case is stepped exactly as ibm_step steps it alone, so
FP32 results are bitwise those of a plain handle (the correction applies its
summed correction itself and the tiles take the vector paths, whose FP32
arithmetic is the scalar paths'); 16-bit storage agrees to its rounding."""
import numpy as np
import pytest

from paper_1803_09380_gb300 import ibm
from paper_1803_09380_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FIELDS = (ibm.FIELD_RHO, ibm.FIELD_UX, ibm.FIELD_UY, ibm.FIELD_BODIES, ibm.FIELD_RESIDUAL)


def _mix():
    """Couette rings, fixed cylinders in channels, settling disks in closed
    boxes (moving bodies: band rebuilt every step), a marker-free box, an MRT
    channel with extrapolation sides, and a ring large enough to need
    several correction CTAs."""
    stream = wl.serving_stream(n_requests=10, seed=11, steps=90, couette_n=(40, 160), cyl_ny=(40, 90),
                               box=(80, 200), disk_d=(10.0, 16.0))
    cases = [(c, s) for _, c, s in stream]
    cases.append((wl.Case("empty", 70, 33, 0.7, bc=(1, 1, 2, 2), wall_u=(0, 0, 0, 0, 0.01, 0, 0, 0)), 37))
    cases.append((wl.paper_cylinder(20.0, diameter=10), 45))
    cases.append((wl.couette(256), 21))                  # 878 markers: two correction CTAs at 512 per CTA
    return cases


def _fields(case):
    return FIELDS if case.bodies else FIELDS[:3] + FIELDS[4:]


def _batched(cases, prec="fp32", **kw):
    kw.setdefault("max_active", 8)
    kw.setdefault("steps_per_launch", 16)
    with ibm.Server(batched=True, **kw) as srv:
        ids = [srv.submit(c, s, prec=prec) for c, s in cases]
        srv.wait()
        st = srv.stats()
        res = [{f: srv.result(i, f) for f in _fields(c)} for i, (c, _) in zip(ids, cases)]
    return res, st


def _alone(case, steps, prec):
    with ibm.Lattice.from_case(case, prec=prec) as lat:
        lat.step(steps)
        r, u, v = lat.moments()
        return {ibm.FIELD_RHO: r, ibm.FIELD_UX: u, ibm.FIELD_UY: v,
                ibm.FIELD_BODIES: lat.bodies, ibm.FIELD_RESIDUAL: lat.resid}


def test_batched_fp32_is_bitwise_a_plain_handle():
    cases = _mix()
    got, st = _batched(cases)
    assert st["completed"] == len(cases) and st["failed"] == 0
    for (c, s), g in zip(cases, got):
        ref = _alone(c, s, "fp32")
        for f in _fields(c):
            assert np.array_equal(g[f], ref[f]), (c.name, f, np.max(np.abs(g[f] - ref[f])))


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_batched_16bit_storage_agrees_with_a_plain_handle(prec):
    cases = _mix()[:6]
    got, st = _batched(cases, prec=prec)
    assert st["failed"] == 0
    for (c, s), g in zip(cases, got):
        ref = _alone(c, s, prec)
        for f in (ibm.FIELD_UX, ibm.FIELD_UY):
            scale = max(np.max(np.abs(ref[f])), 1e-12)
            # the band segments' scalar path of ibm_step rounds f - w_i once
            # more than the vector path: differences at the storage rounding
            assert np.max(np.abs(g[f] - ref[f])) / scale < 2e-2, (c.name, f)


def test_batched_results_are_the_same_alone_and_in_the_mix():
    cases = _mix()
    mixed, _ = _batched(cases, max_active=6, steps_per_launch=12)
    for k in (0, 3, len(cases) - 2):
        alone, _ = _batched([cases[k]], max_active=1, steps_per_launch=7)
        for f in _fields(cases[k][0]):
            assert np.array_equal(alone[0][f], mixed[k][f]), (cases[k][0].name, f)


def test_batched_settings_do_not_change_results():
    cases = _mix()[:7]
    base, _ = _batched(cases, tile_nodes=32768)
    for kw in (dict(tile_nodes=1000, corr_first=2), dict(tile_nodes=4000, ib_markers_per_cta=100)):
        other, _ = _batched(cases, **kw)
        for b, o in zip(base, other):
            for f in b:
                assert np.array_equal(b[f], o[f]), (kw, f)


def test_autotuner_picks_a_candidate_and_keeps_the_statistics_clean():
    sample = [c for c, _ in _mix()[:5]]
    with ibm.Server(batched=True, max_active=8, steps_per_launch=8) as srv:
        t, m, o, sec = srv.autotune(sample, 24, tile_nodes=[2048, 16384], markers_per_cta=[256, 512])
        assert t in (2048, 16384) and m in (256, 512) and o in (1, 2) and sec > 0
        st = srv.stats()
        assert st["submitted"] == 0 and st["completed"] == 0
        i = srv.submit(sample[0], 10)
        srv.wait()
        assert srv.result(i, ibm.FIELD_UX).shape == (sample[0].ny, sample[0].nx)


def test_batched_server_refuses_fp64():
    with ibm.Server(batched=True) as srv:
        with pytest.raises(ibm.IBMError) as e:
            srv.submit(wl.couette(48), 10, prec="fp64")
        assert e.value.status == ibm.IBM_ERR_INVALID
