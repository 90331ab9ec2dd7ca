"""Pins of the FP64 oracle against closed forms and invariants fixed by the
paper (arXiv 1803.09380) and by the mathematics -- never against the oracle
itself.  Each test names the passage it pins and the kind of mistake that
would make it fail."""
import math

import numpy as np
import pytest

import oracle
from paper_1803_09380_gb300 import workloads as wl

# D2Q9 lattice vectors as the rows j_x, j_y of the transform matrix (Eq. 5).
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


# ---------------------------------------------------------------- Eq. 15c
def test_delta4_point_values():
    """Eq. 15c at r = 0, 1, 1.5, 2: 1/2, 1/4, (1 - sqrt(2)/2)/4, 0."""
    assert oracle.delta4(0.0) == 0.5
    assert abs(oracle.delta4(1.0) - 0.25) < 1e-16
    assert abs(oracle.delta4(-1.5) - 0.25 * (1 - math.sqrt(0.5))) < 1e-16
    assert oracle.delta4(2.0) == 0.0
    assert oracle.delta4(2.5) == 0.0


@pytest.mark.parametrize("x0", [0.0, 0.13, 0.5, 0.77, 0.999, 3.4])
def test_delta4_partition_of_unity_and_square_sum(x0):
    """For any offset the 4-point cosine kernel sums to 1 over the integers
    and its squares sum to 3/8 (closed forms of Eq. 15c); a wrong constant,
    width or argument scaling breaks one of them."""
    ks = np.arange(math.floor(x0) - 3, math.floor(x0) + 4)
    d = np.array([oracle.delta4(x0 - k) for k in ks])
    assert abs(d.sum() - 1.0) < 1e-15
    assert abs((d * d).sum() - 3.0 / 8.0) < 1e-15


# ---------------------------------------------------------------- Eqs. 3, 7
@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.03, 0.05, -0.02),
                                       (0.97, -0.08, 0.11)])
def test_equilibrium_moments(rho, ux, uy):
    """Eq. 3 with the weights of Eq. 4: zeroth, first and second moments are
    rho, rho u and rho u u + rho/3 I (c_s^2 = 1/3)."""
    f = oracle.feq(rho, ux, uy)
    assert abs(f.sum() - rho) < 1e-15
    assert abs((EX * f).sum() - rho * ux) < 1e-15
    assert abs((EY * f).sum() - rho * uy) < 1e-15
    assert abs((EX * EX * f).sum() - (rho * ux * ux + rho / 3)) < 1e-15
    assert abs((EX * EY * f).sum() - rho * ux * uy) < 1e-15
    assert abs((EY * EY * f).sum() - (rho * uy * uy + rho / 3)) < 1e-15


def test_moments_match_lattice_vectors():
    """Eq. 7 in the oracle's summation order equals the plain sums over the
    lattice vectors of Eq. 5."""
    p = np.random.default_rng(3).random(9)
    r, jx, jy = oracle.moments(p)
    assert abs(r - p.sum()) < 1e-15
    assert abs(jx - (EX * p).sum()) < 1e-15
    assert abs(jy - (EY * p).sum()) < 1e-15


# ---------------------------------------------------------------- Eqs. 22-28
def _rest_lattice(n, n_corr):
    return oracle.Lattice(n, n, 0.8, n_corr=n_corr)


@pytest.mark.parametrize("y0,xi", [(7.3, 0.37), (8.0, 0.0), (5.91, 0.5)])
def test_straight_line_contracts_by_five_eighths(y0, xi):
    """A periodic straight line of markers at unit spacing (ds = 1) with a
    uniform velocity mismatch U on fluid at rest: one spread followed by one
    interpolation returns 3/8 of the momentum mismatch (partition of unity
    along the line times the 3/8 square sum across it), so the residual of
    Eqs. 22-27 contracts by exactly 5/8 per iteration.  A dropped ds, a
    wrong spreading weight, a sequential (Gauss-Seidel) marker sweep or a
    correction applied to the wrong population fails this."""
    n, N = 16, 10
    L = _rest_lattice(n, N)
    xy = np.stack([np.arange(n) + xi, np.full(n, y0)], axis=1)
    U = (0.01, 0.004)
    L.add_body(xy, 1.0, u=U, xc=(0.0, y0))
    mass0 = L.f.sum()
    L.ib_correct()
    r = L.resid
    mag = math.hypot(*U)
    for k in range(N + 1):
        assert abs(r[k] - mag * (5.0 / 8.0) ** k) < 1e-15 + 1e-12 * mag
    assert abs(L.f.sum() - mass0) < 1e-13 * mass0


@pytest.mark.parametrize("ds", [1.0, 0.5])
def test_isolated_marker_contraction(ds):
    """A single marker: the interpolation of its own spread returns
    (3/8)^2 ds = 9 ds / 64 of the mismatch, so r^n = (1 - 9 ds/64)^n |U|."""
    n, N = 16, 10
    L = _rest_lattice(n, N)
    U = (-0.02, 0.013)
    L.add_body(np.array([[7.3, 8.6]]), ds, u=U, xc=(7.3, 8.6))
    L.ib_correct()
    q = 1.0 - 9.0 * ds / 64.0
    mag = math.hypot(*U)
    for k, rk in enumerate(L.resid):
        assert abs(rk - mag * q ** k) < 1e-13 * mag


def test_correction_conserves_mass_and_matches_eulerian_force():
    """With rho_b = rho* the deviation of Eq. 28 has zero sum over the nine
    directions, so Eq. 27 conserves mass; and the marker-side sum of Eq. 29
    equals the sum of the spread corrections over the Eulerian nodes
    (partition of unity), up to rounding."""
    case = wl.couette_64()
    L = oracle.Lattice(case.nx, case.ny, case.tau, n_corr=case.n_corr)
    for b in case.bodies:
        L.add_body(b.xy, b.ds, **b.as_kwargs())
    L.step(20)
    m0 = L.f.sum()
    L.ib_correct()
    assert abs(L.f.sum() - m0) < 1e-13 * m0
    Fm = L.bodies[:, 6:8].sum(axis=0)
    Fe = L.force_euler
    assert np.all(np.abs(Fm - Fe) < 1e-14 + 1e-10 * np.abs(Fe).max())
    assert np.abs(Fe).max() > 1e-8      # a real force, not a trivial zero


# ---------------------------------------------------------------- rest state
def test_rest_state_stays_exactly_at_rest():
    """All walls at rest and f at the rest equilibrium: with rho_b = rho*
    (Eq. 24) the density parts of f^eq(rho_b, U) and (f^eq)* are the same
    number, and with U = 0 and u = 0 the velocity parts are exactly zero, so
    the deviation of Eq. 28 is exactly zero.  u and the no-slip residual stay
    exactly 0 for 2000 steps and the mirror pairs of populations stay equal
    bit for bit."""
    case = wl.couette(32, wall_speed=0.0)
    L = oracle.Lattice(case.nx, case.ny, case.tau, n_corr=case.n_corr)
    for b in case.bodies:
        L.add_body(b.xy, b.ds, **b.as_kwargs())
    L.step(2000)
    rho, ux, uy = L.moments()
    assert np.all(ux == 0.0) and np.all(uy == 0.0)
    assert np.all(L.resid == 0.0)
    f = L.f
    assert np.array_equal(f[1], f[3]) and np.array_equal(f[2], f[4])
    assert np.array_equal(f[5], f[7]) and np.array_equal(f[6], f[8])
    assert np.all(L.bodies[:, 6:9] == 0.0)


def test_config0_no_slip_residual_contracts():
    """The 64 x 64 ring case (radii 10 and 25, wall speed 0.01, 10
    iterations).  Eqs. 22-27 contract the momentum mismatch of a straight
    line by exactly 5/8 per iteration (pinned above); the rings are close to
    it.  On the first step, from fluid at rest, r^0 is the wall speed and
    r^N / r^0 <= 2 (5/8)^10; over the whole 5000-step run the residual left
    after the 10 iterations stays below 2 (5/8)^10 of the wall speed, and
    each iteration of the first step contracts it."""
    case = wl.couette_64()
    L = oracle.Lattice(case.nx, case.ny, case.tau, n_corr=case.n_corr,
                       threaded=oracle.threaded_available())
    for b in case.bodies:
        L.add_body(b.xy, b.ds, **b.as_kwargs())
    bound = 2.0 * (5.0 / 8.0) ** 10
    L.step(1)
    r = L.resid
    assert abs(r[0] - 0.01) < 1e-15
    assert r[-1] / r[0] <= bound
    assert np.all(np.diff(r) < 0.0)
    worst = r[-1]
    for _ in range(49):
        L.step(100)
        worst = max(worst, L.resid[-1])
    assert worst / 0.01 <= bound


def test_threaded_build_is_bitwise_the_serial_build():
    """The -fopenmp build spreads only loops without a summation order over
    threads: populations, moments, residuals and forces agree bit for bit."""
    if not oracle.threaded_available():
        pytest.skip("gcc -fopenmp is not available")
    oracle.set_threads(4)
    case = wl.settling_pair(nx=48, ny=90, diameter=10.0, density_ratio=1.2, gravity=2e-4)
    out = []
    for threaded in (False, True):
        L = oracle.Lattice(case.nx, case.ny, case.tau, bc=case.bc, n_corr=case.n_corr,
                           threaded=threaded)
        for b in case.bodies:
            L.add_body(b.xy, b.ds, **b.as_kwargs())
        L.step(30)
        out.append((L.f, L.moments()[1], L.resid, L.bodies))
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_mass_conserved_on_couette():
    """BGK collision, periodic streaming and the correction all conserve
    mass: relative drift stays at rounding level."""
    case = wl.couette_64()
    L = oracle.Lattice(case.nx, case.ny, case.tau, n_corr=case.n_corr)
    for b in case.bodies:
        L.add_body(b.xy, b.ds, **b.as_kwargs())
    m0 = L.f.sum()
    L.step(300)
    assert abs(L.f.sum() - m0) < 2e-13 * m0


# ---------------------------------------------------------------- Eqs. 1, 3, 8
def _amplitude(field, axis_len, mode=1):
    """Complex amplitude of sin/cos mode `mode` of a 1-D profile."""
    k = 2 * math.pi * mode * np.arange(axis_len) / axis_len
    s = 2.0 / axis_len * (field * np.sin(k)).sum()
    c = 2.0 / axis_len * (field * np.cos(k)).sum()
    return complex(s, c)


@pytest.mark.parametrize("tau", [0.8, 0.6, 1.2])
def test_shear_wave_decays_at_lattice_viscosity(tau):
    """A shear wave decays as exp(-nu k^2 t) with nu = (tau - 1/2)/3 (Eq. 8,
    c_s^2 = 1/3); the lattice error of the rate is O(k^2) ~ 0.2 % here."""
    nx, ny, T = 4, 128, 600
    L = oracle.Lattice(nx, ny, tau, n_corr=0)
    rho, ux, uy = wl.shear_wave(nx, ny, amplitude=1e-3)
    L.init_equilibrium(rho, ux, uy)
    L.step(T)
    _, ux, _ = L.moments()
    a = abs(_amplitude(ux[:, 0], ny))
    nu = (tau - 0.5) / 3.0
    k = 2 * math.pi / ny
    # moments are taken before the collision of step T, i.e. after T-1 steps
    rate = -math.log(a / 1e-3) / (T - 1)
    assert abs(rate / (nu * k * k) - 1.0) < 0.01


def test_wave_is_advected_by_the_mean_flow():
    """A transverse wave u_y(x) on a uniform stream U0 translates with U0:
    its phase moves by k U0 t.  A streaming step with a wrong direction
    sign, or a collision that breaks Galilean invariance at first order,
    fails."""
    nx, ny, T, U0 = 64, 4, 300, 0.05
    L = oracle.Lattice(nx, ny, 0.8, n_corr=0)
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    k = 2 * math.pi / nx
    ux = np.full((ny, nx), U0)
    uy = 1e-3 * np.sin(k * x)
    L.init_equilibrium(np.ones((ny, nx)), ux, uy)
    L.step(T)
    _, _, uy = L.moments()
    a = _amplitude(uy[0], nx)
    phase = math.atan2(-a.imag, a.real)     # sin(k (x - s)) has this phase
    expected = k * U0 * (T - 1)
    assert abs(phase - expected) < 0.02 * expected


# ---------------------------------------------------------------- walls
def test_bounceback_moving_wall_gives_exact_linear_couette():
    """Half-way bounce-back with a moving top wall: the steady plane Couette
    profile is linear between walls at y = -1/2 and y = ny - 1/2, and
    half-way bounce-back reproduces linear profiles exactly."""
    nx, ny, Uw = 4, 8, 0.02
    wall_u = np.zeros(8)
    wall_u[6] = Uw                          # +y side moves along x
    L = oracle.Lattice(nx, ny, 1.0, bc=(0, 0, 1, 1), wall_u=wall_u, n_corr=0)
    L.step(3000)
    _, ux, uy = L.moments()
    y = np.arange(ny)
    exact = Uw * (y + 0.5) / ny
    assert np.max(np.abs(ux[:, 0] - exact)) < 1e-11
    assert np.max(np.abs(uy)) < 1e-14


def test_freeslip_walls_keep_neumann_mode():
    """Free-slip (specular) walls at y = -1/2 and ny - 1/2 admit the mode
    u_x = A cos(pi (y + 1/2) / ny), which decays at nu (pi/ny)^2; bounce-back
    there would force u_x -> 0 at the walls and decay much faster."""
    nx, ny, T, tau = 4, 64, 800, 0.8
    L = oracle.Lattice(nx, ny, tau, bc=(0, 0, 2, 2), n_corr=0)
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    prof = np.cos(math.pi * (y + 0.5) / ny)
    L.init_equilibrium(np.ones((ny, nx)), 1e-3 * prof, np.zeros((ny, nx)))
    L.step(T)
    _, ux, _ = L.moments()
    a = (ux[:, 0] * prof[:, 0]).sum() / (prof[:, 0] ** 2).sum()
    nu = (tau - 0.5) / 3.0
    rate = -math.log(a / 1e-3) / (T - 1)
    assert abs(rate / (nu * (math.pi / ny) ** 2) - 1.0) < 0.02


def test_inlet_outlet_keep_uniform_stream():
    """An equilibrium inlet at U_in, a zero-gradient outlet and free-slip
    side walls keep a uniform stream at U_in exactly steady."""
    nx, ny, U = 32, 12, 0.05
    L = oracle.Lattice(nx, ny, 0.8, bc=(3, 4, 2, 2), inlet_u=(U, 0.0), n_corr=0)
    L.init_equilibrium(np.ones((ny, nx)), np.full((ny, nx), U), np.zeros((ny, nx)))
    L.step(200)
    rho, ux, uy = L.moments()
    assert np.max(np.abs(ux - U)) < 1e-13
    assert np.max(np.abs(uy)) < 1e-13
    assert np.max(np.abs(rho - 1.0)) < 1e-13


def test_outlet_lets_a_pulse_leave():
    """A density pulse launched toward the zero-gradient outlet leaves the
    domain instead of reflecting back fully: the remaining excess mass falls
    well below what a closed wall would keep."""
    nx, ny = 64, 4
    def run(bc):
        L = oracle.Lattice(nx, ny, 0.8, bc=bc, n_corr=0)
        x = np.arange(nx)[None, :] * np.ones((ny, 1))
        rho = 1.0 + 1e-3 * np.exp(-((x - 50.0) / 3.0) ** 2)
        L.init_equilibrium(rho, np.zeros((ny, nx)), np.zeros((ny, nx)))
        L.step(120)
        r, _, _ = L.moments()
        return (r - 1.0).sum()
    open_excess = run((1, 4, 0, 0))
    closed_excess = run((1, 1, 0, 0))
    assert open_excess < 0.6 * closed_excess


# ---------------------------------------------------------------- Eqs. 37-42
def test_free_fall_without_fluid_force_follows_recurrence():
    """With no hydrodynamic force (no correction iterations), Eqs. 37, 40-42
    with the lagged internal-mass term give du^n = r du^{n-1} + (1 - r) g,
    r = rho_f/rho_s, so du^n = g (1 - r^(n+1)) and
    x^{n+1} = x^n + u^n + du^n / 2."""
    L = oracle.Lattice(32, 32, 0.8, n_corr=0)
    b = wl.disk(16.0, 16.0, 6.0, 1.5, 1e-4)
    L.add_body(b.xy, b.ds, **b.as_kwargs())
    g = -1e-4
    r = 1.0 / 1.5
    u, y = 0.0, 16.0
    for n in range(12):
        L.ib_correct()
        L.move_bodies()
        du = g * (1 - r ** (n + 1))
        y, u = y + u + 0.5 * du, u + du
        B = L.bodies[0]
        assert abs(B[3] - u) < 1e-17 + 1e-12 * abs(u)
        assert abs(B[1] - y) < 1e-12
    # markers moved rigidly with the centre
    assert np.allclose(L.markers[:, 1] - L.bodies[0, 1], b.xy[:, 1] - 16.0, atol=1e-12)


def test_collision_force_of_eq39():
    """Two touching disks (gap 0) at rest, no gravity in the force balance
    other than the scale c = M (1 - rho_f/rho_s) |g|: Eq. 39 gives
    c/eps ((d - R_i - R_j - xi)/xi)^2 = c/eps = 100 c along the centre line."""
    L = oracle.Lattice(64, 64, 0.8, n_corr=0)
    D, ratio, g = 8.0, 2.0, 1e-4
    a = wl.disk(30.0, 32.0, D, ratio, g)
    b = wl.disk(38.0, 32.0, D, ratio, g)
    a.gravity = b.gravity = (0.0, -g)
    L.add_body(a.xy, a.ds, **a.as_kwargs())
    L.add_body(b.xy, b.ds, **b.as_kwargs())
    L.ib_correct()
    L.move_bodies()
    M = ratio * math.pi * D * D / 4
    c = M * (1 - 1 / ratio) * g
    B = L.bodies
    # u^1 = F_tot / M with F_tot = F_c + M (1 - 1/ratio) g_vec
    assert abs(B[0, 2] * M - (-100.0 * c)) < 1e-12 * c
    assert abs(B[1, 2] * M - (100.0 * c)) < 1e-12 * c
    assert abs(B[0, 3] * M - (-c)) < 1e-12 * c
