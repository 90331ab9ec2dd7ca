"""Checkpoint and resume through the C ABI: IBM_FIELD_F plus
IBM_FIELD_BODY_STATE written into a fresh lattice made with the same
parameters and bodies continue the run bit for bit (FP64 and FP32 storage).

The settling pair exercises free bodies (pose, velocities and the previous
step's velocities of the internal-mass terms, Eqs. 37-38; markers moved
rigidly and the band rebuilt on restore) in a bounce-back box; the
checkpoint is taken after an odd number of steps, so the populations are
read out of the swapped AA layout and written back in the natural one.
The Couette rings are fixed bodies with prescribed wall velocity."""
import numpy as np
import pytest

from paper_1803_09380_gb300 import ibm
from paper_1803_09380_gb300 import workloads as wl

from _helpers import gpu_lattice

pytestmark = pytest.mark.gpu


def _pair():
    return wl.settling_pair(nx=64, ny=130, diameter=10.0, density_ratio=1.2, gravity=2e-4)


def _state(lat):
    return (lat.f, lat.bodies, lat.read(ibm.FIELD_BODY_STATE), lat.markers, lat.resid, lat.moments()[1])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case_name,before,after", [("settling_pair", 151, 120), ("couette64", 40, 61)])
def test_resume_from_a_checkpoint_is_bitwise(prec, case_name, before, after):
    case = _pair() if case_name == "settling_pair" else wl.couette(64)
    a = gpu_lattice(case, prec, None)
    a.step(before)
    ck = a.checkpoint()
    b = gpu_lattice(case, prec, None)
    b.step(3)                       # a lattice that has run elsewhere: its state is overwritten
    b.restore(ck)
    a.step(after)
    b.step(after)
    for x, y in zip(_state(a), _state(b)):
        assert np.array_equal(x, y)
    a.close()
    b.close()


def test_body_state_round_trip_and_argument_errors():
    case = _pair()
    lat = gpu_lattice(case, "fp64", None)
    lat.step(20)
    st = lat.read(ibm.FIELD_BODY_STATE)
    assert st.shape == (2, 9)
    # the state is the pose and velocities of BODIES, plus the previous step's velocities
    assert np.array_equal(st[:, :6], lat.bodies[:, :6])
    lat.write(ibm.FIELD_BODY_STATE, st)
    assert np.array_equal(lat.read(ibm.FIELD_BODY_STATE), st)
    with pytest.raises(ibm.IBMError):
        ibm.ibm_write_fields(lat.h, ibm.FIELD_BODY_STATE, st[:1])
    bad = st.copy()
    bad[0, 4] = np.nan
    with pytest.raises(ibm.IBMError):
        lat.write(ibm.FIELD_BODY_STATE, bad)
    # a failed write changed nothing
    assert np.array_equal(lat.read(ibm.FIELD_BODY_STATE), st)
    lat.close()


def test_moving_a_body_by_its_state_moves_its_markers():
    """Writing a pose moves the markers rigidly (Eqs. 41-42): a shift of the
    centre shifts every marker of that body by the same amount."""
    case = _pair()
    lat = gpu_lattice(case, "fp64", None)
    lat.step(2)
    st = lat.read(ibm.FIELD_BODY_STATE)
    m0 = lat.markers
    st[0, 0] += 3.0
    st[0, 1] -= 5.0
    lat.write(ibm.FIELD_BODY_STATE, st)
    m1 = lat.markers
    n0 = len(case.bodies[0].xy)
    assert np.allclose(m1[:n0] - m0[:n0], [3.0, -5.0], atol=1e-12)
    assert np.array_equal(m1[n0:], m0[n0:])
    lat.step(5)                     # the band follows the moved markers
    assert np.all(np.isfinite(lat.f))
    lat.close()
