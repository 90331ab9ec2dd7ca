"""Pins of the oracle's body motion and of the signs of its force and torque
(arXiv 1803.09380, Eqs. 24, 29, 37-42), against closed forms and the
direction the correction must push: rigid rotation counter-clockwise for
positive omega, uniform motion without force or torque, the first residual
of a rigidly moving boundary in fluid at rest, and hydrodynamic force and
torque that oppose the motion."""
import math

import numpy as np
import pytest

import oracle
from paper_1803_09380_gb300 import workloads as wl


def _ring_body(L, xc, radius, kind, u=(0.0, 0.0), omega=0.0, count=None):
    xy, ds = wl.ring(xc[0], xc[1], radius, count=count)
    vol = math.pi * radius * radius
    L.add_body(xy, ds, kind=kind, xc=xc, u=u, omega=omega, rho_s=1.5, rho_f=1.0,
               volume=vol, inertia=1.5 * vol * radius * radius / 2.0, radius=radius)
    return xy


def test_prescribed_motion_rotates_markers_counter_clockwise():
    """A prescribed body translates by u and turns by omega every step; a
    marker that starts at angle 0 is at angle n omega (positive =
    counter-clockwise): after a quarter turn it sits straight above the
    centre."""
    L = oracle.Lattice(64, 64, 0.8, n_corr=0)
    xc, R, u, om = (20.0, 24.0), 6.0, (0.1, -0.05), math.pi / 40.0
    xy = _ring_body(L, xc, R, oracle.BODY_PRESCRIBED, u=u, omega=om, count=16)
    assert abs(xy[0, 0] - (xc[0] + R)) < 1e-12 and abs(xy[0, 1] - xc[1]) < 1e-12
    for _ in range(20):
        L.move_bodies()
    B = L.bodies[0]
    cx, cy = xc[0] + 20 * u[0], xc[1] + 20 * u[1]
    assert abs(B[0] - cx) < 1e-12 and abs(B[1] - cy) < 1e-12
    assert abs(B[5] - math.pi / 2) < 1e-12
    m = L.markers
    assert abs(m[0, 0] - cx) < 1e-11 and abs(m[0, 1] - (cy + R)) < 1e-11
    # every marker keeps its distance to the centre
    assert np.allclose(np.hypot(m[:, 0] - cx, m[:, 1] - cy), R, atol=1e-11)


def test_free_body_without_force_or_torque_moves_uniformly():
    """Eqs. 37-42 with no hydrodynamic force (no correction iterations), no
    gravity and no history impulse: u and omega stay, x^n = x^0 + n u and
    theta^n = n omega."""
    L = oracle.Lattice(64, 64, 0.8, n_corr=0)
    xc, u, om = (30.0, 30.0), (0.02, -0.01), 0.01
    _ring_body(L, xc, 5.0, oracle.BODY_FREE, u=u, omega=om)
    for _ in range(15):
        L.ib_correct()
        L.move_bodies()
    B = L.bodies[0]
    assert abs(B[0] - (xc[0] + 15 * u[0])) < 1e-12
    assert abs(B[1] - (xc[1] + 15 * u[1])) < 1e-12
    assert abs(B[2] - u[0]) < 1e-15 and abs(B[3] - u[1]) < 1e-15
    assert abs(B[4] - om) < 1e-15 and abs(B[5] - 15 * om) < 1e-12


@pytest.mark.parametrize("u,om", [((0.0, 0.0), 0.004), ((0.01, -0.02), 0.0), ((0.01, 0.005), 0.003)])
def test_first_residual_is_the_boundary_speed_in_fluid_at_rest(u, om):
    """In fluid at rest the interpolated momentum is zero and rho* = 1
    (partition of unity), so r^0 = max_l |U_l| with U_l = u + omega x
    (X_l - x_c) (Eq. 24), which on a ring of radius R is
    max_l |u + omega R t_l| for the tangents t_l."""
    L = oracle.Lattice(48, 48, 0.8, n_corr=4)
    xc, R = (24.0, 23.7), 6.0
    xy = _ring_body(L, xc, R, oracle.BODY_PRESCRIBED, u=u, omega=om)
    L.ib_correct()
    U = np.stack([u[0] - om * (xy[:, 1] - xc[1]), u[1] + om * (xy[:, 0] - xc[0])], axis=1)
    expect = np.max(np.hypot(U[:, 0], U[:, 1]))
    assert abs(L.resid[0] - expect) < 1e-13


def test_torque_opposes_rotation_and_fluid_turns_with_the_body():
    """A disk turning counter-clockwise in fluid at rest: the correction
    gives the fluid counter-clockwise momentum, so the torque on the body
    (Eq. 29) is negative, the net force vanishes by symmetry, and next to
    the rightmost marker the fluid moves in +y."""
    L = oracle.Lattice(64, 64, 0.8, n_corr=10)
    xc, R, om = (32.0, 32.0), 8.0, 0.004
    _ring_body(L, xc, R, oracle.BODY_PRESCRIBED, omega=om, count=64)
    L.step(1)
    F = L.bodies[0, 6:9]
    assert F[2] < 0
    assert abs(F[0]) < 1e-9 * abs(F[2]) / R and abs(F[1]) < 1e-9 * abs(F[2]) / R
    rho, ux, uy = L.moments()
    assert uy[32, 40] > 0 and uy[32, 24] < 0 and ux[40, 32] < 0 and ux[24, 32] > 0


def test_drag_opposes_translation():
    """A disk moving in +x through fluid at rest: the correction pushes the
    fluid along +x, so the force on the body is along -x and has no y part
    (the set-up is symmetric about y = y_c)."""
    L = oracle.Lattice(64, 64, 0.8, n_corr=10)
    xc, R, U = (32.0, 32.0), 8.0, 0.01
    _ring_body(L, xc, R, oracle.BODY_PRESCRIBED, u=(U, 0.0), count=64)
    L.step(1)
    F = L.bodies[0, 6:9]
    assert F[0] < 0
    assert abs(F[1]) < 1e-9 * abs(F[0]) and abs(F[2]) < 1e-9 * abs(F[0]) * R
    rho, ux, uy = L.moments()
    # the fluid at the boundary, inside and outside, is dragged along
    assert ux[39, 32] > 0 and ux[41, 32] > 0 and ux[23, 32] > 0 and ux[25, 32] > 0


@pytest.mark.parametrize("rho0,u0", [(1.0, (0.03, -0.02)), (1.02, (-0.01, 0.015))])
def test_boundary_moving_with_a_uniform_stream_needs_no_correction(rho0, u0):
    """Galilean consistency of Eqs. 22-28: in a uniform equilibrium stream
    (rho0, u0), a boundary whose markers move with u0 already satisfies the
    no-slip condition.  The interpolated equilibria equal f^eq(rho0, u0)
    and rho* = rho0 (partition of unity), so every deviation, residual,
    force and torque vanishes and f is left as it was (to rounding)."""
    L = oracle.Lattice(48, 48, 0.8, n_corr=10)
    L.init_equilibrium(rho0, u0[0], u0[1])
    f0 = L.f
    _ring_body(L, (24.0, 23.6), 6.5, oracle.BODY_PRESCRIBED, u=u0)
    L.ib_correct()
    # rounding level: a wrong target or interpolation would give O(|u0|) = 1e-2
    assert np.max(np.abs(L.resid)) < 1e-14
    assert np.max(np.abs(L.f - f0)) < 1e-14
    assert np.max(np.abs(L.bodies[0, 6:9])) < 1e-12
