"""The largest lattice the ABI accepts: ny = 65535 rows and nx * ny just
under 2^31 nodes (FP16 storage, about 72 GB on the device), which puts
every population index above 2^32.  A small ring far from the edges, two
steps: the correction residuals and the body force and torque equal those
of the same ring on a 256 x 256 lattice at the same offset within a
128-node span (two steps carry nothing further than a few nodes, and every
sum of the method is in a fixed order).  The marker coordinates differ in
magnitude (about 19200 against 128), so their FP64 rounding differs in the
last bits: the comparison allows 1e-6 relative, far below any indexing
error, which would change the result entirely."""
import math

import numpy as np
import pytest

from paper_1803_09380_gb300 import ibm
from paper_1803_09380_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _ring_case(lat, cx, cy):
    xy, ds = wl.ring(cx, cy, 10.3, count=64)
    lat.add_markers(xy, ds, xc=(cx, cy), omega=0.01 / 10.3, radius=10.3)


def test_largest_lattice_matches_a_small_one():
    torch = pytest.importorskip("torch")
    nx, ny = 32768, 65535
    assert nx * ny < 2 ** 31
    free, _ = torch.cuda.mem_get_info()
    if free < 90e9:
        pytest.skip("needs about 80 GB of free device memory")
    results = []
    for (n_x, n_y, cx, cy) in ((256, 256, 128.37, 128.61), (nx, ny, 128.0 * 150 + 0.37, 40000.61)):
        lat = ibm.Lattice(n_x, n_y, 0.8, prec="fp16")
        _ring_case(lat, cx, cy)
        lat.step(2, ibm.STEP_NO_MACRO)
        results.append((lat.resid.copy(), lat.bodies[:, 6:9].copy()))
        lat.close()
        del lat
        torch.cuda.empty_cache()
    (r0, f0), (r1, f1) = results
    assert np.all(np.isfinite(r1)) and r1[0] > 0
    np.testing.assert_allclose(r1, r0, rtol=1e-6, atol=0)
    np.testing.assert_allclose(f1, f0, rtol=1e-6, atol=1e-12)
