"""Pins of the oracle's 2- and 3-point delta functions (arXiv 1803.09380,
Eq. 15a, b) and of the correction loop run with them."""
import math

import numpy as np
import pytest

import oracle


def _window(fn, x0):
    ks = np.arange(math.floor(x0) - 3, math.floor(x0) + 4)
    return ks, np.array([fn(x0 - k) for k in ks])


def test_point_values():
    assert oracle.delta2(0.0) == 1.0 and oracle.delta2(0.25) == 0.75 and oracle.delta2(1.0) == 0.0
    assert abs(oracle.delta3(0.0) - 2.0 / 3.0) < 1e-16
    assert abs(oracle.delta3(1.0) - 1.0 / 6.0) < 1e-16
    assert abs(oracle.delta3(0.5) - 0.5) < 1e-16          # the two branches meet at 1/2
    assert oracle.delta3(1.5) == 0.0 and oracle.delta3(-1.7) == 0.0


@pytest.mark.parametrize("x0", [0.0, 0.13, 0.5, 0.77, 0.999, 3.4])
def test_partition_of_unity_and_first_moment(x0):
    """Both kernels sum to 1 over the integers and have zero first moment
    for any offset (the interpolation is exact for linear fields)."""
    for fn in (oracle.delta2, oracle.delta3):
        ks, d = _window(fn, x0)
        assert abs(d.sum() - 1.0) < 1e-15
        assert abs(((x0 - ks) * d).sum()) < 1e-15


@pytest.mark.parametrize("x0", [0.0, 0.21, 0.5, 0.86])
def test_square_sums(x0):
    """The 3-point kernel's squares sum to 1/2 for every offset; the hat's
    to (1 - e)^2 + e^2 with e the fractional offset."""
    _, d3 = _window(oracle.delta3, x0)
    assert abs((d3 * d3).sum() - 0.5) < 1e-15
    _, d2 = _window(oracle.delta2, x0)
    e = x0 - math.floor(x0)
    assert abs((d2 * d2).sum() - ((1 - e) ** 2 + e ** 2)) < 1e-15


@pytest.mark.parametrize("points,y0", [(3, 7.3), (3, 8.0), (2, 7.3), (2, 5.5)])
def test_straight_line_contraction(points, y0):
    """A periodic straight line of markers at unit spacing contracts the
    residual by 1 - sum_k delta(y0 - k)^2 per iteration: 1/2 for the
    3-point kernel, 1 - (1 - e)^2 - e^2 for the hat."""
    n, N = 16, 8
    L = oracle.Lattice(n, n, 0.8, n_corr=N, delta_points=points)
    xy = np.stack([np.arange(n) + 0.37, np.full(n, y0)], axis=1)
    U = (0.01, -0.006)
    L.add_body(xy, 1.0, u=U, xc=(0.0, y0))
    L.ib_correct()
    e = y0 - math.floor(y0)
    q = 0.5 if points == 3 else 1.0 - (1 - e) ** 2 - e ** 2
    mag = math.hypot(*U)
    for k, rk in enumerate(L.resid):
        assert abs(rk - mag * q ** k) < 1e-15 + 1e-12 * mag
