"""One particle settling in a channel (arXiv 1803.09380, section 3.3.1):
the paper reports that the particle drifts to the channel centre line for
every density ratio, and that at the larger ratios (1.01, 1.03) it
overshoots and oscillates about it before settling there.  The paper prints
no numbers for this case (its Fig. 8 compares curves), so these tests check
that behaviour.  Setup: workloads.paper_settling (D = 26 lattice units,
W = 4D, tau = 0.6, gravity from the physical scales, zero-velocity
extrapolation inlet behind the particle, free outflow ahead), FP32, 40,000
steps (about 2 s of physical time)."""
import numpy as np
import pytest

from paper_1803_09380_gb300 import ibm
from paper_1803_09380_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _trajectory(ratio, steps=40000, every=200):
    case = wl.paper_settling(ratio)
    lat = ibm.Lattice.from_case(case, prec="fp32")
    W = case.meta["width"]
    tr = []
    for _ in range(steps // every):
        lat.step(every, flags=ibm.STEP_NO_MACRO)
        b = lat.bodies[0]
        tr.append(((b[1] - W / 2.0) / W, b[2], b[3]))
    return case, np.array(tr)


def test_heavier_particle_overshoots_then_settles_on_the_centre_line():
    _, tr = _trajectory(1.03)
    off, u, v = tr[:, 0], tr[:, 1], tr[:, 2]
    assert off[0] > 0.3
    assert off.min() < -0.02                    # crosses the centre line
    assert (v > 0).any() and (v < 0).any()      # the lateral velocity changes sign
    assert abs(off[-1]) < 0.02                  # and ends on the centre line
    assert u[-1] > 0 and abs(u[-1] / u[-10] - 1) < 0.01   # at its terminal velocity


def test_lighter_particle_drifts_toward_the_centre_line():
    _, tr = _trajectory(1.01)
    off = tr[:, 0]
    assert off[-1] < 0.5 * off[0]
    assert np.all(np.diff(off[5:]) < 1e-4)      # monotonic approach so far
