"""Pins of the oracle's MRT collision (arXiv 1803.09380, Eqs. 2, 5, 6) against
closed forms fixed by the moment basis, not against the oracle itself."""
import math

import numpy as np
import pytest

import oracle
from paper_1803_09380_gb300 import workloads as wl

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
PAPER_RATES = (1.1, 1.25, 1.8)     # s_e, s_eps, s_q of section 3


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.03, 0.07, -0.04), (0.91, -0.11, 0.09)])
def test_equilibrium_moments_have_their_closed_forms(rho, ux, uy):
    """M f^eq for the equilibrium of Eq. 3 gives the textbook equilibrium
    moments of the D2Q9 basis: e = rho(-2 + 3u^2), eps = rho(1 - 3u^2),
    q = -rho u, p_xx = rho(ux^2 - uy^2), p_xy = rho ux uy.  A wrong sign or
    entry in a row of Eq. 5 changes one of them."""
    m = oracle.mrt_matrix() @ oracle.feq(rho, ux, uy)
    u2 = ux * ux + uy * uy
    want = [rho, rho * (-2 + 3 * u2), rho * (1 - 3 * u2), rho * ux, -rho * ux,
            rho * uy, -rho * uy, rho * (ux * ux - uy * uy), rho * ux * uy]
    np.testing.assert_allclose(m, want, rtol=0, atol=1e-15)


def test_rows_are_orthogonal_with_the_usual_norms():
    """The basis of Eq. 5 is orthogonal; |row|^2 = 9, 36, 36, 6, 12, 6, 12,
    4, 4.  The collision inverts M through this property."""
    M = oracle.mrt_matrix()
    np.testing.assert_array_equal(M @ M.T, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4]).astype(float))


def test_mrt_with_equal_rates_is_bgk():
    """S = I / tau turns Eq. 2 into the single-relaxation operator."""
    rng = np.random.default_rng(3)
    for tau in (0.53, 0.8, 1.7):
        p = oracle.feq(1.0, 0.05, -0.02) + 1e-3 * rng.standard_normal(9)
        fe = oracle.feq(*_macro(p))
        got = oracle.mrt_collide(np.full(9, 1.0 / tau), p, fe)
        np.testing.assert_allclose(got, p - (p - fe) / tau, rtol=0, atol=2e-16)


def _macro(p):
    rho = p.sum()
    return rho, (EX * p).sum() / rho, (EY * p).sum() / rho


def test_each_moment_relaxes_by_its_own_rate():
    """After one collision the non-equilibrium part of moment k is scaled by
    1 - s_k (Eq. 2 in moment space), with the rates in the row order of
    Eq. 6: a rate placed on the wrong moment fails."""
    rng = np.random.default_rng(11)
    s = np.array([0.3, 1.1, 1.25, 0.7, 1.8, 0.9, 1.6, 1.4, 0.6])
    M = oracle.mrt_matrix()
    for _ in range(5):
        p = oracle.feq(1.0, 0.03, 0.01) + 1e-2 * rng.standard_normal(9)
        fe = oracle.feq(1.0, 0.02, -0.01)
        ps = oracle.mrt_collide(s, p, fe)
        np.testing.assert_allclose(M @ (ps - fe), (1 - s) * (M @ (p - fe)), rtol=0, atol=1e-15)


def test_collision_conserves_mass_and_momentum():
    rng = np.random.default_rng(5)
    s = np.array([1.25, *PAPER_RATES[:2], 1.25, PAPER_RATES[2], 1.25, PAPER_RATES[2], 1.25, 1.25])
    for _ in range(5):
        p = oracle.feq(1.0, 0.04, -0.03) + 1e-3 * rng.standard_normal(9)
        ps = oracle.mrt_collide(s, p, oracle.feq(*_macro(p)))
        assert abs(ps.sum() - p.sum()) < 1e-15
        assert abs((EX * ps).sum() - (EX * p).sum()) < 1e-15
        assert abs((EY * ps).sum() - (EY * p).sum()) < 1e-15


def _amplitude(field, n):
    k = 2 * math.pi * np.arange(n) / n
    return math.hypot(2.0 / n * (field * np.sin(k)).sum(), 2.0 / n * (field * np.cos(k)).sum())


@pytest.mark.parametrize("tau,rates", [(0.8, PAPER_RATES), (0.6, PAPER_RATES), (0.8, (1.5, 1.4, 1.2))])
def test_shear_wave_decay_is_set_by_the_stress_rate(tau, rates):
    """A shear wave decays at nu = (tau - 1/2)/3 (Eq. 8) whatever the other
    rates: only the stress moments p_xx, p_xy carry shear viscosity."""
    nx, ny, T = 4, 128, 600
    L = oracle.Lattice(nx, ny, tau, n_corr=0, mrt=rates)
    L.init_equilibrium(*wl.shear_wave(nx, ny, amplitude=1e-3))
    L.step(T)
    _, ux, _ = L.moments()
    rate = -math.log(_amplitude(ux[:, 0], ny) / 1e-3) / (T - 1)
    nu = (tau - 0.5) / 3.0
    assert abs(rate / (nu * (2 * math.pi / ny) ** 2) - 1.0) < 0.01


def test_energy_rate_changes_sound_damping_only():
    """A longitudinal (sound) wave is damped through the energy moment too,
    so changing s_e changes its decay while a shear wave is unaffected to
    the lattice error."""
    nx, ny, T = 128, 4, 400

    def sound(rates):
        L = oracle.Lattice(nx, ny, 0.8, n_corr=0, mrt=rates)
        x = np.arange(nx)[None, :] * np.ones((ny, 1))
        rho = 1.0 + 1e-4 * np.cos(2 * math.pi * x / nx)
        L.init_equilibrium(rho, np.zeros((ny, nx)), np.zeros((ny, nx)))
        L.step(T)
        r, _, _ = L.moments()
        return np.abs(r[0] - r[0].mean()).max()

    a_lo, a_hi = sound((0.6, 1.25, 1.8)), sound((1.6, 1.25, 1.8))
    assert a_lo < 0.9 * a_hi       # smaller s_e: larger bulk viscosity, more damping
