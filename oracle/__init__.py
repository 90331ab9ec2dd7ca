"""Plain FP64 CPU oracle of the distribution-function-correction IB-LBM.

TEST INFRASTRUCTURE ONLY: the slow, obviously-correct restatement of the
method (arXiv 1803.09380, section 2, Eqs. 1-8, 15c, 22-29; section 3.3,
Eqs. 37-42) that the CUDA library is checked against.  Only the tests, the
package smoke check and the CPU-baseline leg of the benchmark may import this
module.  It shares no code with the CUDA library: the arithmetic lives in
``ibm_oracle.c``, this file only compiles it with gcc and marshals arrays.

Parity status of the functions (what pins each one is in ``tests/``):
  delta4, feq, moments            pinned by closed forms (partition of unity,
                                  sum of squares 3/8, equilibrium moments)
  delta2, delta3 (Eq. 15a, b)     pinned by partition of unity, zero first
                                  moment, sum of squares (1/2 for delta3) and
                                  the straight-line contraction 1 - sum d^2
  IB correction loop              pinned by the straight-line 5/8 contraction
                                  and the isolated-marker 1 - 9/64 contraction
  collide + stream (periodic)     pinned by the shear-wave decay rate and
                                  Galilean advection of the wave
  walls (bounce-back, free-slip)  pinned by plane Poiseuille / plug flow
  inlet / outlet                  pinned by uniform-flow preservation
  extrapolation inlet / outlet    pinned by uniform-flow preservation, the
                                  exact rebuild of an equilibrium neighbour
                                  and plane Poiseuille flow
  whole step                      pinned by the analytic Couette profile
                                  (Eq. 34) and its measured convergence slope
  MRT collision (Eqs. 2, 5, 6)    pinned by the closed-form equilibrium
                                  moments, reduction to BGK at equal rates,
                                  per-moment relaxation factors 1 - s_k and
                                  the shear-wave decay set by 1/tau alone
  Newton-Euler body update        pinned by closed-form free fall with no
                                  fluid force (Eqs. 40-42), uniform motion
                                  without force or torque, prescribed rigid
                                  motion (counter-clockwise for omega > 0),
                                  Eq. 39 at contact
  marker velocity, force, torque  pinned by the first residual of a moving
                                  boundary in fluid at rest (= max |U_l|,
                                  Eq. 24), mass conservation and Eulerian =
                                  Lagrangian force (Eq. 29), and drag and
                                  torque that oppose the motion
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ibm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_OMP_PATH = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_libs: dict = {}

PERIODIC, BOUNCEBACK, FREESLIP, INLET_EQ, OUTLET_ZEROGRAD = 0, 1, 2, 3, 4
INLET_NEE, OUTLET_NEE = 5, 6
BODY_FIXED, BODY_PRESCRIBED, BODY_FREE = 0, 1, 2

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)

_CFLAGS = ["-O2", "-ffp-contract=off", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared"]


def _compile(path: str, extra: list, force: bool) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *_CFLAGS, *extra, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile ibm_oracle.c into oracle/_build/liboracle.so (plain gcc, FP64,
    no contraction into fused multiply-adds, one thread), and the same source
    with -fopenmp into liboracle_omp.so when the compiler supports it."""
    path = _compile(_LIB_PATH, [], force)
    try:
        _compile(_OMP_PATH, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        pass                      # the threaded build is optional
    return path


def _declare(lib):
    vp = ctypes.c_void_p
    lib.ora_delta4.restype = ctypes.c_double
    lib.ora_delta4.argtypes = [ctypes.c_double]
    for name in ("ora_delta2", "ora_delta3"):
        getattr(lib, name).restype = ctypes.c_double
        getattr(lib, name).argtypes = [ctypes.c_double]
    lib.ora_set_delta.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.ora_set_reading.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 4
    lib.ora_set_threads.restype = ctypes.c_int
    lib.ora_set_threads.argtypes = [ctypes.c_int]
    lib.ora_set_marker_velocities.restype = ctypes.c_int
    lib.ora_set_marker_velocities.argtypes = [ctypes.c_void_p, _D, ctypes.c_int]
    lib.ora_feq.argtypes = [ctypes.c_double] * 3 + [_D]
    lib.ora_moments.argtypes = [_D, _D, _D, _D]
    lib.ora_create.restype = vp
    lib.ora_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                               ctypes.c_double, _I, _D, _D, ctypes.c_int]
    lib.ora_destroy.argtypes = [vp]
    lib.ora_add_body.restype = ctypes.c_int
    lib.ora_add_body.argtypes = [vp, ctypes.c_int, _D, _D, _D, ctypes.c_int]
    for name in ("ora_ib_correct", "ora_move_bodies", "ora_record_moments",
                 "ora_collide_stream", "ora_open_boundaries"):
        getattr(lib, name).argtypes = [vp]
    lib.ora_step.argtypes = [vp, ctypes.c_int]
    for name in ("ora_get_f", "ora_set_f", "ora_get_resid", "ora_get_bodies",
                 "ora_get_markers", "ora_get_force_euler"):
        getattr(lib, name).argtypes = [vp, _D]
    lib.ora_init_equilibrium.argtypes = [vp, _D, _D, _D]
    lib.ora_get_moments.argtypes = [vp, _D, _D, _D]
    lib.ora_num_markers.restype = ctypes.c_int
    lib.ora_num_markers.argtypes = [vp]
    lib.ora_num_bodies.restype = ctypes.c_int
    lib.ora_num_bodies.argtypes = [vp]
    lib.ora_set_mrt.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.ora_mrt_matrix.argtypes = [_D]
    lib.ora_mrt_collide.argtypes = [_D, _D, _D, _D]


def _load(threaded: bool = False):
    """The serial library, or the -fopenmp build when ``threaded``."""
    with _lock:
        key = "omp" if threaded else "serial"
        if key in _libs:
            return _libs[key]
        build()
        if threaded and not os.path.exists(_OMP_PATH):
            raise RuntimeError("the threaded oracle build (gcc -fopenmp) is not available")
        if threaded:
            # idle threads sleep instead of spinning: the oracle shares the
            # host with other work (tests, the GPU driver thread)
            os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")
        lib = ctypes.CDLL(_OMP_PATH if threaded else _LIB_PATH)
        _declare(lib)
        _libs[key] = lib
        return lib


def threaded_available() -> bool:
    build()
    return os.path.exists(_OMP_PATH)


def set_threads(n: int) -> int:
    """Threads of the threaded build (0: all host cores); returns the count
    it will use."""
    return int(_load(True).ora_set_threads(int(n)))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def delta4(r: float) -> float:
    """Eq. 15c, 4-point cosine delta function."""
    return _load().ora_delta4(float(r))


def delta2(r: float) -> float:
    """Eq. 15a: the 2-point delta function."""
    return _load().ora_delta2(float(r))


def delta3(r: float) -> float:
    """Eq. 15b: the 3-point delta function."""
    return _load().ora_delta3(float(r))


def feq(rho: float, ux: float, uy: float) -> np.ndarray:
    """Eq. 3 equilibrium of the nine D2Q9 populations."""
    out = np.zeros(9)
    _load().ora_feq(rho, ux, uy, _dp(out))
    return out


def moments(p) -> tuple[float, float, float]:
    """Eq. 7: (rho, rho u_x, rho u_y) of nine populations."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    r, jx, jy = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().ora_moments(_dp(p), ctypes.byref(r), ctypes.byref(jx), ctypes.byref(jy))
    return r.value, jx.value, jy.value


def mrt_matrix() -> np.ndarray:
    """The transform matrix M of Eq. 5 as the oracle holds it."""
    out = np.empty((9, 9))
    _load().ora_mrt_matrix(_dp(out))
    return out


def mrt_collide(rates, p, fe) -> np.ndarray:
    """One MRT collision (Eq. 2) at one node: p - M^-1 S M (p - fe) with
    S = diag(rates) (Eq. 6, nine rates in the row order of Eq. 5)."""
    s = np.ascontiguousarray(rates, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    fe = np.ascontiguousarray(fe, dtype=np.float64)
    out = np.empty(9)
    _load().ora_mrt_collide(_dp(s), _dp(p), _dp(fe), _dp(out))
    return out


# Alternative readings of section 2.3 that ora_set_reading can switch on (the
# default, all off: nodal equilibria interpolated, rho_b = rho*, correction of
# the post-stream populations, spreading weighted by ds).
READINGS = ("interp_moments", "rho_b_ref", "post_collision", "unit_ds")


class Lattice:
    """One oracle lattice: D2Q9 BGK with immersed bodies, all FP64.
    ``mrt=(s_e, s_eps, s_q)`` switches the collision to MRT (Eqs. 2, 5, 6)
    with the stress moments relaxing at 1/tau.

    ``threaded`` runs the -fopenmp build (bitwise the same results; thread
    count from ``set_threads`` or OMP_NUM_THREADS).  ``reading`` switches on
    alternative readings of section 2.3 by name (see READINGS).

    ``bc`` gives the rule of the four sides (-x, +x, -y, +y); ``wall_u`` the
    velocity of each side as a moving bounce-back wall; ``inlet_u`` the inflow
    velocity of an inlet on the -x side.  f starts at the rest equilibrium.
    """

    def __init__(self, nx, ny, tau, rho0=1.0, bc=(0, 0, 0, 0), wall_u=None,
                 inlet_u=(0.0, 0.0), n_corr=10, mrt=None, delta_points=4,
                 threaded=False, reading=None):
        self._lib = _load(threaded)
        self.nx, self.ny, self.n_corr = int(nx), int(ny), int(n_corr)
        bc_a = (ctypes.c_int * 4)(*[int(b) for b in bc])
        wu = np.zeros(8) if wall_u is None else np.ascontiguousarray(wall_u, dtype=np.float64).reshape(8)
        iu = np.ascontiguousarray(inlet_u, dtype=np.float64)
        self._h = self._lib.ora_create(self.nx, self.ny, float(tau), float(rho0),
                                       bc_a, _dp(wu), _dp(iu), self.n_corr)
        if not self._h:
            raise MemoryError("oracle lattice allocation failed")
        if mrt is not None:
            self._lib.ora_set_mrt(self._h, *[float(v) for v in mrt])
        if delta_points not in (2, 3, 4):
            raise ValueError("delta_points must be 2, 3 or 4 (Eq. 15a-c)")
        self._lib.ora_set_delta(self._h, int(delta_points))
        if reading:
            unknown = set(reading) - set(READINGS)
            if unknown:
                raise ValueError(f"unknown readings {sorted(unknown)}")
            self._lib.ora_set_reading(self._h, *[int(bool(reading.get(k, 0))) for k in READINGS])

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ora_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    # ---- bodies
    def add_body(self, xy, ds, kind=BODY_FIXED, xc=(0.0, 0.0), u=(0.0, 0.0),
                 omega=0.0, theta=0.0, rho_s=1.0, rho_f=1.0, volume=0.0,
                 inertia=0.0, radius=0.0, gravity=(0.0, 0.0)) -> int:
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        ds = np.ascontiguousarray(np.broadcast_to(ds, (xy.shape[0],)), dtype=np.float64)
        bd = np.array([xc[0], xc[1], u[0], u[1], omega, theta, rho_s, rho_f,
                       volume, inertia, radius, gravity[0], gravity[1]], dtype=np.float64)
        return self._lib.ora_add_body(self._h, int(kind), _dp(bd), _dp(xy), _dp(ds),
                                      xy.shape[0])

    def set_marker_velocities(self, uv):
        """Prescribed U_l of every marker of a fixed body, (M, 2) array,
        from the next step on."""
        uv = np.ascontiguousarray(uv, dtype=np.float64).reshape(-1, 2)
        if self._lib.ora_set_marker_velocities(self._h, _dp(uv), uv.shape[0]) != 0:
            raise ValueError("one velocity pair per marker is required")

    # ---- stepping
    def step(self, n=1):
        self._lib.ora_step(self._h, int(n))

    def ib_correct(self):
        self._lib.ora_ib_correct(self._h)

    def move_bodies(self):
        self._lib.ora_move_bodies(self._h)

    def open_boundaries(self):
        self._lib.ora_open_boundaries(self._h)

    def record_moments(self):
        self._lib.ora_record_moments(self._h)

    def collide_stream(self):
        self._lib.ora_collide_stream(self._h)

    # ---- state
    @property
    def f(self) -> np.ndarray:
        out = np.empty((9, self.ny, self.nx))
        self._lib.ora_get_f(self._h, _dp(out))
        return out

    @f.setter
    def f(self, value):
        a = np.ascontiguousarray(value, dtype=np.float64).reshape(9, self.ny, self.nx)
        self._lib.ora_set_f(self._h, _dp(a))

    def init_equilibrium(self, rho, ux, uy):
        shp = (self.ny, self.nx)
        r = np.ascontiguousarray(np.broadcast_to(rho, shp), dtype=np.float64)
        a = np.ascontiguousarray(np.broadcast_to(ux, shp), dtype=np.float64)
        b = np.ascontiguousarray(np.broadcast_to(uy, shp), dtype=np.float64)
        self._lib.ora_init_equilibrium(self._h, _dp(r), _dp(a), _dp(b))

    def moments(self):
        """(rho, u_x, u_y) of the last corrected pre-collision state."""
        r = np.empty((self.ny, self.nx)); a = np.empty_like(r); b = np.empty_like(r)
        self._lib.ora_get_moments(self._h, _dp(r), _dp(a), _dp(b))
        return r, a, b

    @property
    def resid(self) -> np.ndarray:
        out = np.empty(self.n_corr + 1)
        self._lib.ora_get_resid(self._h, _dp(out))
        return out

    @property
    def bodies(self) -> np.ndarray:
        """Per body: xc, yc, ux, uy, omega, theta, Fx, Fy, T."""
        nb = self._lib.ora_num_bodies(self._h)
        out = np.empty((nb, 9))
        if nb:
            self._lib.ora_get_bodies(self._h, _dp(out))
        return out

    @property
    def markers(self) -> np.ndarray:
        nm = self._lib.ora_num_markers(self._h)
        out = np.empty((nm, 2))
        if nm:
            self._lib.ora_get_markers(self._h, _dp(out))
        return out

    @property
    def force_euler(self) -> np.ndarray:
        out = np.empty(2)
        self._lib.ora_get_force_euler(self._h, _dp(out))
        return out
