"""Pins of the oracle's non-equilibrium-extrapolation inlet and outlet (the
boundary scheme section 3.2 uses for the cylinder channel) against exact
solutions, not against the oracle itself."""
import numpy as np
import pytest

import oracle

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
NEE = (oracle.INLET_NEE, oracle.OUTLET_NEE)


def test_uniform_stream_is_kept_exactly():
    """A uniform stream at the inlet velocity and the outlet density is a
    fixed point: f is the same equilibrium everywhere, the rebuilt columns
    equal it, and collision and streaming leave it unchanged."""
    nx, ny, U = 40, 12, (0.05, 0.0)
    L = oracle.Lattice(nx, ny, 0.7, bc=NEE + (oracle.FREESLIP, oracle.FREESLIP), inlet_u=U, n_corr=0)
    L.init_equilibrium(np.ones((ny, nx)), np.full((ny, nx), U[0]), np.zeros((ny, nx)))
    L.step(150)
    rho, ux, uy = L.moments()
    assert np.abs(rho - 1).max() < 1e-13
    assert np.abs(ux - U[0]).max() < 1e-13 and np.abs(uy).max() < 1e-13


def test_equilibrium_neighbour_is_rebuilt_as_the_boundary_equilibrium():
    """If the inner neighbour is at equilibrium, its non-equilibrium part is
    zero and the boundary node becomes f^eq(rho_f, U_in) at the inlet and
    f^eq(rho0, u_f) at the outlet."""
    nx, ny = 10, 5
    U = (0.04, -0.01)
    L = oracle.Lattice(nx, ny, 0.9, bc=NEE + (oracle.PERIODIC, oracle.PERIODIC), inlet_u=U, n_corr=0)
    rng = np.random.default_rng(2)
    rho = 1 + 0.02 * rng.standard_normal((ny, nx))
    ux = 0.03 * rng.standard_normal((ny, nx))
    uy = 0.03 * rng.standard_normal((ny, nx))
    L.init_equilibrium(rho, ux, uy)
    L.open_boundaries()
    f = L.f
    for y in range(ny):
        np.testing.assert_allclose(f[:, y, 0], oracle.feq(rho[y, 1], *U), rtol=0, atol=1e-15)
        np.testing.assert_allclose(f[:, y, nx - 1], oracle.feq(1.0, ux[y, nx - 2], uy[y, nx - 2]),
                                   rtol=0, atol=1e-15)


def test_non_equilibrium_part_is_carried_over():
    """A perturbed neighbour: the boundary node's deviation from its own
    equilibrium is the neighbour's deviation from the neighbour's (the
    extrapolated non-equilibrium part), and the boundary density and
    velocity come out as prescribed."""
    nx, ny, U = 8, 4, (0.06, 0.0)
    L = oracle.Lattice(nx, ny, 0.8, bc=NEE + (oracle.PERIODIC, oracle.PERIODIC), inlet_u=U, n_corr=0)
    L.init_equilibrium(np.ones((ny, nx)), np.full((ny, nx), 0.02), np.zeros((ny, nx)))
    f = L.f + 1e-3 * np.random.default_rng(5).standard_normal((9, ny, nx))
    L.f = f
    L.open_boundaries()
    g = L.f
    for y in range(ny):
        p = f[:, y, 1]
        rf = p.sum()
        uf = ((EX * p).sum() / rf, (EY * p).sum() / rf)
        b = g[:, y, 0]
        rb = b.sum()
        assert abs(rb - rf) < 1e-15                         # rho_b = rho(x_f)
        assert abs((EX * b).sum() / rb - U[0]) < 1e-14      # u_b = U_in
        np.testing.assert_allclose(b - oracle.feq(rf, *U), p - oracle.feq(rf, *uf), rtol=0, atol=1e-16)


def test_channel_develops_plane_poiseuille_flow():
    """A uniform inflow between half-way bounce-back walls develops into the
    parabola u(y) ~ 1 - (2 s / H)^2 (s from the centre line, H = ny), and in
    the steady state the mass flux sum_y rho u is the same at every column
    of the channel."""
    nx, ny, U, tau = 120, 15, 0.02, 0.8
    L = oracle.Lattice(nx, ny, tau, bc=NEE + (oracle.BOUNCEBACK, oracle.BOUNCEBACK), inlet_u=(U, 0.0),
                       n_corr=0)
    L.init_equilibrium(np.ones((ny, nx)), np.full((ny, nx), U), np.zeros((ny, nx)))
    L.step(5000)
    rho, ux, uy = L.moments()
    s = np.arange(ny) + 0.5 - ny / 2.0
    shape = 1 - (2 * s / ny) ** 2
    got = ux[:, 90]
    assert np.abs(got / got.mean() - shape / shape.mean()).max() < 1e-2
    q = (rho * ux).sum(axis=0)[1:nx - 1]
    assert np.abs(q / q.mean() - 1).max() < 1e-5
    assert np.abs(uy[:, 90]).max() < 1e-4 * U
