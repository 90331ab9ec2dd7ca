"""Seeded synthetic inputs shaped like the paper's cases.

This module holds geometry, configuration numbers and seeded random draws
only -- none of the method's arithmetic (no equilibria, no delta function, no
collision).  Both the CUDA library's tests and the oracle's tests take their
inputs from here, so neither side computes the other's inputs.

Cases (arXiv 1803.09380):
  * cylindrical Couette flow, section 3.1.2 (Eqs. 32-34): two concentric
    rings of Lagrangian markers, the inner one rotating;
  * flow past a fixed cylinder, section 3.2: one ring in a channel with an
    equilibrium inlet, zero-gradient outlet and free-slip side walls;
  * settling disks, section 3.3 (Eqs. 37-42): free rings in a closed box.
Markers are spaced about one lattice unit apart along each ring; the arc
length per marker is the ring perimeter over the marker count (Eq. 26).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PERIODIC, BOUNCEBACK, FREESLIP, INLET_EQ, OUTLET_ZEROGRAD = 0, 1, 2, 3, 4
INLET_NEE, OUTLET_NEE = 5, 6   # non-equilibrium extrapolation sides
BODY_FIXED, BODY_PRESCRIBED, BODY_FREE = 0, 1, 2


@dataclass
class Body:
    xy: np.ndarray            # (M, 2) marker positions, lattice units
    ds: np.ndarray            # (M,) arc length per marker
    kind: int = BODY_FIXED
    xc: tuple = (0.0, 0.0)
    u: tuple = (0.0, 0.0)
    omega: float = 0.0
    theta: float = 0.0
    rho_s: float = 1.0
    rho_f: float = 1.0
    volume: float = 0.0
    inertia: float = 0.0
    radius: float = 0.0
    gravity: tuple = (0.0, 0.0)

    def as_kwargs(self) -> dict:
        return dict(kind=self.kind, xc=self.xc, u=self.u, omega=self.omega,
                    theta=self.theta, rho_s=self.rho_s, rho_f=self.rho_f,
                    volume=self.volume, inertia=self.inertia, radius=self.radius,
                    gravity=self.gravity)


@dataclass
class Case:
    name: str
    nx: int
    ny: int
    tau: float
    rho0: float = 1.0
    bc: tuple = (PERIODIC,) * 4
    wall_u: tuple = (0.0,) * 8
    inlet_u: tuple = (0.0, 0.0)
    n_corr: int = 10
    bodies: list = field(default_factory=list)
    mrt: tuple | None = None  # None: BGK; else MRT rates (s_e, s_eps, s_q), Eq. 6
    delta_points: int = 4     # delta function of Eq. 15: 2, 3 or 4 points
    meta: dict = field(default_factory=dict)

    @property
    def n_markers(self) -> int:
        return sum(b.xy.shape[0] for b in self.bodies)


def ring(xc: float, yc: float, radius: float, count: int | None = None,
         phase: float = 0.0):
    """Markers on a circle at angles 2 pi l / M + phase, M = round(2 pi R)
    unless given; returns (xy, ds) with ds = 2 pi R / M."""
    m = int(round(2.0 * math.pi * radius)) if count is None else int(count)
    ang = 2.0 * math.pi * np.arange(m) / m + phase
    xy = np.stack([xc + radius * np.cos(ang), yc + radius * np.sin(ang)], axis=1)
    ds = np.full(m, 2.0 * math.pi * radius / m)
    return xy, ds


def couette(n: int, r1: float | None = None, r2: float | None = None,
            wall_speed: float = 0.01, tau: float = 0.8, n_corr: int = 10,
            center: tuple | None = None) -> Case:
    """Cylindrical Couette flow on an n x n periodic lattice: inner ring of
    radius r1 (default 0.156 n) turning with tangential speed ``wall_speed``,
    outer ring of radius r2 (default 0.39 n) at rest (section 3.1.2)."""
    r1 = 0.156 * n if r1 is None else float(r1)
    r2 = 0.39 * n if r2 is None else float(r2)
    cx, cy = (n / 2.0, n / 2.0) if center is None else center
    xy1, ds1 = ring(cx, cy, r1)
    xy2, ds2 = ring(cx, cy, r2)
    inner = Body(xy1, ds1, BODY_FIXED, xc=(cx, cy), omega=wall_speed / r1, radius=r1)
    outer = Body(xy2, ds2, BODY_FIXED, xc=(cx, cy), omega=0.0, radius=r2)
    return Case(f"couette{n}", n, n, tau, n_corr=n_corr, bodies=[inner, outer],
                meta=dict(r1=r1, r2=r2, cx=cx, cy=cy, wall_speed=wall_speed))


def couette_64() -> Case:
    """The 64 x 64 case with radii 10 and 25 centred at (32, 32)."""
    return couette(64, 10.0, 25.0, center=(32.0, 32.0))


def couette_analytic(case: Case, x: np.ndarray, y: np.ndarray):
    """Eq. 34 for the Couette case: steady (u_x, u_y) at points (x, y);
    rigid rotation inside r1 and rest outside r2 (the fictitious fluid)."""
    m = case.meta
    r1, r2, U = m["r1"], m["r2"], m["wall_speed"]
    dx, dy = x - m["cx"], y - m["cy"]
    r = np.hypot(dx, dy)
    w1 = U / r1
    R = r1 / r2
    with np.errstate(divide="ignore", invalid="ignore"):
        ut = (r1 ** 2 - R ** 2 * r ** 2) * w1 / ((1.0 - R ** 2) * r)
    ut = np.where(r < r1, w1 * r, np.where(r > r2, 0.0, ut))
    with np.errstate(divide="ignore", invalid="ignore"):
        sx = np.where(r > 0, -dy / r, 0.0)
        sy = np.where(r > 0, dx / r, 0.0)
    return ut * sx, ut * sy


def couette_paper(r2: float, ratio: float, tau: float, re: float = 10.0,
                  mrt: bool = True, n_corr: int = 10) -> Case:
    """Cylindrical Couette flow as section 3.1.2 sets it up: outer radius r2
    lattice units (the grid spacing is 1/r2 of the outer radius), radius
    ratio R = r1/r2, relaxation time tau and Re = U1 (r2 - r1)/nu = 10 held
    fixed under refinement, so the wall speed U1 = Re nu/(r2 - r1) falls as
    the grid is refined (nu = (tau - 1/2)/3).  The MRT rates of section 3.
    The periodic box leaves four nodes between the outer ring and its image."""
    r1 = ratio * r2
    nu = (tau - 0.5) / 3.0
    u1 = re * nu / (r2 - r1)
    n = int(round(2 * r2)) + 8
    c = couette(n, r1, r2, wall_speed=u1, tau=tau, n_corr=n_corr, center=(n / 2.0, n / 2.0))
    c.name = f"couette_paper_R{ratio:g}_tau{tau:g}_r{r2:g}"
    c.mrt = (1.1, 1.25, 1.8) if mrt else None
    c.meta.update(re=re, ratio=ratio, nu=nu)
    return c


def paper_cylinder(re: float, diameter: int = 40, u0: float = 0.1, mrt: bool = True,
                   n_corr: int = 10) -> Case:
    """Flow past a fixed cylinder as section 3.2 sets it up: a 40D x 20D
    channel, the cylinder at (10D, 10D), D = 40 lattice units, inflow
    U0 = 0.1 through a non-equilibrium-extrapolation inlet, a free outflow
    through an extrapolation outlet, free-slip side walls (the paper does
    not say), the MRT rates of section 3 and tau from Re = U0 D / nu."""
    nu = u0 * diameter / re
    tau = 0.5 + 3.0 * nu
    c = (10.0 * diameter, 10.0 * diameter + 0.3)
    markers = int(round(math.pi * diameter))
    xy, ds = ring(c[0], c[1], diameter / 2.0, count=markers)
    body = Body(xy, ds, BODY_FIXED, xc=c, radius=diameter / 2.0)
    return Case(f"cylinder_re{re:g}_d{diameter}", 40 * diameter, 20 * diameter, tau,
                bc=(INLET_NEE, OUTLET_NEE, FREESLIP, FREESLIP), inlet_u=(u0, 0.0), n_corr=n_corr,
                bodies=[body], mrt=(1.1, 1.25, 1.8) if mrt else None,
                meta=dict(diameter=diameter, u_in=u0, re=re))


def paper_settling(density_ratio: float, diameter: int = 26, tau: float = 0.6,
                   drop: float = 3.0) -> Case:
    """One particle settling in a channel (section 3.3.1), laid along x: the
    channel is 4D wide (bounce-back walls at the y sides) and 400/13 D long,
    the particle (D = 0.1 cm on 26 lattice units) starts 0.31 W off the
    centre line, `drop` diameters below the zero-velocity inlet at -x, and
    falls toward the free outlet at +x.  Fluid: 1 g/cm^3, nu = 0.01 cm^2/s,
    |g| = 980 cm/s^2, tau = 0.6; the lattice spacing and time step follow
    from D and tau, which fix g in lattice units."""
    d_phys, nu_phys, g_phys = 0.1, 0.01, 980.0
    dx = d_phys / diameter
    nu = (tau - 0.5) / 3.0
    dt = nu * dx * dx / nu_phys
    g = g_phys * dt * dt / dx
    width = 4 * diameter
    length = int(round(400.0 / 13.0 * diameter))
    b = disk(drop * diameter, width / 2.0 + 0.31 * width, float(diameter), density_ratio, g)
    b.gravity = (g, 0.0)
    return Case(f"settle_channel_{density_ratio:g}", length, width, tau,
                bc=(INLET_NEE, OUTLET_NEE, BOUNCEBACK, BOUNCEBACK), inlet_u=(0.0, 0.0), bodies=[b],
                meta=dict(diameter=diameter, dx_cm=dx, dt_s=dt, g=g, width=width))


def taylor_green(L: int, re: float = 10.0, tau: float = 0.65, n_corr: int = 10,
                 markers: int | None = None) -> Case:
    """Taylor-Green vortices with an artificial cylinder (section 3.1.1): a
    periodic 2L x 2L lattice whose node i sits at x = i + 1/2 - L (the
    vortex field of Eq. 30 has period 2L), a cylinder of diameter L at the
    centre whose markers follow Eq. 30, Re = u0 L / nu (10) and tau (0.65)
    fixing u0.  Marker velocities change every step: see taylor_green_fields."""
    nu = (tau - 0.5) / 3.0
    u0 = re * nu / L
    c = L - 0.5
    xy, ds = ring(c, c, L / 2.0, count=markers)
    body = Body(xy, ds, BODY_FIXED, xc=(c, c), radius=L / 2.0)
    return Case(f"tgv{L}", 2 * L, 2 * L, tau, n_corr=n_corr, bodies=[body],
                meta=dict(L=L, u0=u0, nu=nu, center=c, re=re))


def taylor_green_fields(case: Case, x, y, t: float):
    """Eq. 30 at lattice coordinates (x, y) and time t: (rho, u_x, u_y).
    Readings of the garbled print: u_y = +u0 sin(kx) cos(ky) (the printed
    sign gives a divergent field) and the density of the standard vortex
    pressure, rho = rho0 - 3 u0^2/4 (cos 2kx + cos 2ky) e^{-4 nu k^2 t}
    (p = c_s^2 rho), with k = pi / L and rho0 = 1."""
    m = case.meta
    k = math.pi / m["L"]
    X = np.asarray(x, dtype=np.float64) - m["center"]
    Y = np.asarray(y, dtype=np.float64) - m["center"]
    d = math.exp(-2.0 * m["nu"] * k * k * t)
    ux = -m["u0"] * np.cos(k * X) * np.sin(k * Y) * d
    uy = m["u0"] * np.sin(k * X) * np.cos(k * Y) * d
    rho = 1.0 - 0.75 * m["u0"] ** 2 * (np.cos(2 * k * X) + np.cos(2 * k * Y)) * d * d
    return rho, ux, uy


def taylor_green_steps(case: Case) -> int:
    """Time steps to t* = t u0 / L = 1."""
    return int(round(case.meta["L"] / case.meta["u0"]))


def cylinder(nx: int = 1600, ny: int = 800, diameter: float = 40.0,
             center: tuple = (400.0, 400.0), u_in: float = 0.05,
             re: float = 20.0, markers: int = 126, n_corr: int = 10) -> Case:
    """Flow past a fixed cylinder: equilibrium inlet at -x, zero-gradient
    outlet at +x, free-slip walls at +-y; tau from Re = U D / nu with the
    lattice viscosity nu = (tau - 1/2) / 3 (Eq. 8)."""
    nu = u_in * diameter / re
    tau = 0.5 + 3.0 * nu
    xy, ds = ring(center[0], center[1], diameter / 2.0, count=markers)
    body = Body(xy, ds, BODY_FIXED, xc=center, radius=diameter / 2.0)
    return Case(f"cylinder{nx}x{ny}_re{re:g}", nx, ny, tau,
                bc=(INLET_EQ, OUTLET_ZEROGRAD, FREESLIP, FREESLIP),
                inlet_u=(u_in, 0.0), n_corr=n_corr, bodies=[body],
                meta=dict(diameter=diameter, u_in=u_in, re=re))


def disk(xc: float, yc: float, diameter: float, density_ratio: float,
         gravity: float, kind: int = BODY_FREE) -> Body:
    """A free rigid disk (section 3.3): area V = pi D^2 / 4, mass rho_s V,
    moment of inertia M D^2 / 8, fluid density 1, gravity along -y."""
    r = diameter / 2.0
    xy, ds = ring(xc, yc, r)
    vol = math.pi * diameter ** 2 / 4.0
    mass = density_ratio * vol
    return Body(xy, ds, kind, xc=(xc, yc), rho_s=density_ratio, rho_f=1.0,
                volume=vol, inertia=mass * diameter ** 2 / 8.0, radius=r,
                gravity=(0.0, -gravity))


def settling_single(nx: int = 200, ny: int = 600, diameter: float = 20.0,
                    density_ratio: float = 1.5, gravity: float = 2.0e-5,
                    tau: float = 0.8) -> Case:
    """One disk settling in a closed bounce-back box."""
    b = disk(nx / 2.0 + 0.1 * diameter, ny - 3.0 * diameter, diameter,
             density_ratio, gravity)
    return Case(f"settle1_{nx}x{ny}", nx, ny, tau, bc=(BOUNCEBACK,) * 4,
                bodies=[b], meta=dict(diameter=diameter))


def settling_pair(nx: int = 200, ny: int = 800, diameter: float = 20.0,
                  density_ratio: float = 1.01, gravity: float = 1.0e-4,
                  tau: float = 0.8) -> Case:
    """Two disks stacked 2 D apart with a 0.1 D lateral offset (drafting,
    kissing, tumbling)."""
    top = disk(nx / 2.0 - 0.1 * diameter, ny - 4.0 * diameter, diameter,
               density_ratio, gravity)
    low = disk(nx / 2.0, ny - 6.0 * diameter, diameter, density_ratio, gravity)
    return Case(f"settle2_{nx}x{ny}", nx, ny, tau, bc=(BOUNCEBACK,) * 4,
                bodies=[top, low], meta=dict(diameter=diameter))


def shear_wave(nx: int, ny: int, amplitude: float = 0.01, mode: int = 1,
               background=(0.0, 0.0)):
    """Macroscopic fields of a shear wave u_x(y) = A sin(2 pi k y / ny) on a
    uniform background: returns (rho, u_x, u_y) arrays of shape (ny, nx)."""
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    ux = background[0] + amplitude * np.sin(2.0 * math.pi * mode * y / ny)
    uy = np.full((ny, nx), float(background[1]))
    rho = np.ones((ny, nx))
    return rho, ux, uy


def random_fields(nx: int, ny: int, seed: int, du: float = 0.02,
                  drho: float = 0.01):
    """Seeded random smooth-ish macroscopic fields around rest."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + drho * rng.standard_normal((ny, nx))
    ux = du * rng.standard_normal((ny, nx))
    uy = du * rng.standard_normal((ny, nx))
    return rho, ux, uy


def random_perturbation(nx: int, ny: int, seed: int, amplitude: float = 1e-3):
    """Seeded random array of shape (9, ny, nx) to add to populations."""
    rng = np.random.default_rng(seed)
    return amplitude * rng.standard_normal((9, ny, nx))


def serving_stream(n_requests: int = 512, seed: int = 1803, rate_hz: float = 200.0,
                   steps: int = 1000, couette_n=(64, 2048), cyl_ny=(200, 800),
                   cyl_re=(10.0, 100.0), box=(200, 600), disk_d=(10.0, 30.0)):
    """A seeded request stream: Poisson arrivals at rate_hz, families drawn
    uniformly from {Couette with N log-uniform in couette_n, fixed cylinder
    with Re uniform in cyl_re on lattices 2 ny x ny (ny in cyl_ny, D = ny/20),
    one or two settling disks with D uniform in disk_d in a box}; every
    request runs `steps` time steps.  Returns [(arrival_s, Case, steps)]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        fam = int(rng.integers(0, 3))
        if fam == 0:
            n = int(round(math.exp(rng.uniform(math.log(couette_n[0]), math.log(couette_n[1])))))
            n = max(32, n)
            case = couette(n)
        elif fam == 1:
            ny = int(rng.integers(cyl_ny[0] // 10, cyl_ny[1] // 10 + 1)) * 10
            d = ny / 20.0
            case = cylinder(nx=2 * ny, ny=ny, diameter=d, center=(ny / 2.0, ny / 2.0 + 0.3),
                            u_in=0.05, re=float(rng.uniform(*cyl_re)),
                            markers=max(16, int(round(math.pi * d))))
        else:
            nx, ny = box
            d = float(rng.uniform(*disk_d))
            bodies = [disk(nx / 2.0 + 0.1 * d, ny - 3.0 * d, d, 1.2, 1e-4)]
            if rng.random() < 0.5:
                bodies.append(disk(nx / 2.0, ny - 5.5 * d, d, 1.2, 1e-4))
            case = Case(f"settle_{len(bodies)}", nx, ny, 0.8, bc=(BOUNCEBACK,) * 4, bodies=bodies,
                        meta=dict(diameter=d))
        out.append((t, case, steps))
    return out
