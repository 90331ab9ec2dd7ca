"""Thin Python binding of the C ABI in include/ibm.h (argument marshalling
only; every step of the method runs in the CUDA kernels of libibm.so).

The functions carry the ABI's names.  Arrays are numpy FP64 on the host.
There is no fallback: if libibm.so cannot be loaded (not built, or no CUDA
runtime) the first call raises.  With PyTorch present, device memory comes
from PyTorch's caching allocator and work is enqueued on a PyTorch stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

# Kernels on different streams overlap only when they reach the GPU through
# different hardware work queues; CUDA gives a process 8 unless this is set
# before the process creates its CUDA context.  The serving layer keeps
# dozens of lattices (two streams each) resident, so ask for 32.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

IBM_OK, IBM_ERR_INVALID, IBM_ERR_NOMEM, IBM_ERR_CUDA = 0, 1, 2, 3
IBM_ERR_BOUNDS, IBM_ERR_DIVERGED, IBM_ERR_TIMEOUT, IBM_WARN_NOT_CONVERGED = 4, 5, 6, 7
IBM_FP64, IBM_FP32, IBM_FP16_DEV, IBM_BF16_DEV = 0, 1, 2, 3
PERIODIC, BOUNCEBACK, FREESLIP, INLET_EQ, OUTLET_ZEROGRAD = 0, 1, 2, 3, 4
INLET_NEE, OUTLET_NEE = 5, 6   # non-equilibrium extrapolation inlet / outlet
BODY_FIXED, BODY_PRESCRIBED, BODY_FREE = 0, 1, 2
COLL_BGK, COLL_MRT = 0, 1
PAPER_MRT_RATES = (1.1, 1.25, 1.8)   # s_e, s_eps, s_q of section 3
FIELD_RHO, FIELD_UX, FIELD_UY, FIELD_F = 1, 2, 3, 4
FIELD_BODIES, FIELD_RESIDUAL, FIELD_MARKERS, FIELD_MACRO_INIT = 5, 6, 7, 8
FIELD_BODY_STATE = 9
STEP_DEFAULT, STEP_NO_GRAPH, STEP_TIME_KERNELS, STEP_NO_MACRO = 0, 1, 2, 4

PRECISIONS = {"fp64": IBM_FP64, "fp32": IBM_FP32, "fp16": IBM_FP16_DEV, "bf16": IBM_BF16_DEV}

_STATUS = {0: "IBM_OK", 1: "IBM_ERR_INVALID", 2: "IBM_ERR_NOMEM", 3: "IBM_ERR_CUDA",
           4: "IBM_ERR_BOUNDS", 5: "IBM_ERR_DIVERGED", 6: "IBM_ERR_TIMEOUT",
           7: "IBM_WARN_NOT_CONVERGED"}

SYMBOLS = ("ibm_create_lattice", "ibm_add_markers", "ibm_step", "ibm_read_fields",
           "ibm_write_fields", "ibm_sync", "ibm_kernel_times", "ibm_get_sizes",
           "ibm_get_counters", "ibm_destroy", "ibm_last_error", "ibm_set_allocator",
           "ibm_abi_version", "ibm_ib_correct_noalloc", "ibm_set_option",
           "ibm_server_create", "ibm_server_submit", "ibm_server_progress", "ibm_server_wait",
           "ibm_server_result", "ibm_server_release", "ibm_server_get_stats", "ibm_server_destroy",
           "ibm_server_last_error", "ibm_set_marker_velocities", "ibm_autotune_ib",
           "ibm_server_autotune")
IBM_OPT_IB_CTAS, IBM_OPT_IB_THREADS = 1, 2
IBM_OPT_WATCHDOG_STEPS, IBM_OPT_BARRIER_LIMIT_US, IBM_OPT_TEST_DROP_ARRIVAL = 3, 4, 5
IBM_OPT_IB_PHASES = 6
OUT_MACRO, OUT_BODIES, OUT_RESIDUAL = 1, 2, 4


class IBMError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {message}")
        self.status = status


class LatticeDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("tau", ctypes.c_double),
                ("rho0", ctypes.c_double), ("prec", ctypes.c_int), ("bc", ctypes.c_int * 4),
                ("wall_u", (ctypes.c_double * 2) * 4), ("inlet_u", ctypes.c_double * 2),
                ("n_corr", ctypes.c_int), ("corr_tol", ctypes.c_double),
                ("delta_points", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
                ("device", ctypes.c_int), ("collision", ctypes.c_int),
                ("mrt_s", ctypes.c_double * 3)]


class BodyDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("xc", ctypes.c_double * 2), ("u", ctypes.c_double * 2),
                ("omega", ctypes.c_double), ("theta", ctypes.c_double),
                ("rho_s", ctypes.c_double), ("rho_f", ctypes.c_double),
                ("volume", ctypes.c_double), ("inertia", ctypes.c_double),
                ("radius", ctypes.c_double), ("gravity", ctypes.c_double * 2)]


class ServerDesc(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("max_device_bytes", ctypes.c_double),
                ("max_active", ctypes.c_int), ("steps_per_launch", ctypes.c_int),
                ("ib_cta_budget", ctypes.c_int), ("ib_markers_per_cta", ctypes.c_int),
                ("batched", ctypes.c_int), ("tile_nodes", ctypes.c_int), ("corr_first", ctypes.c_int)]


class CaseDesc(ctypes.Structure):
    _fields_ = [("lattice", LatticeDesc), ("nbodies", ctypes.c_int),
                ("bodies", ctypes.POINTER(BodyDesc)), ("nmarkers", ctypes.POINTER(ctypes.c_int)),
                ("xy", ctypes.POINTER(ctypes.c_double)), ("ds", ctypes.POINTER(ctypes.c_double)),
                ("nsteps", ctypes.c_int), ("outputs", ctypes.c_uint)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("active", ctypes.c_longlong), ("pending", ctypes.c_longlong),
                ("failed", ctypes.c_longlong), ("p50_ms", ctypes.c_double),
                ("p95_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("solves_per_s", ctypes.c_double),
                ("mlups", ctypes.c_double), ("device_bytes", ctypes.c_double),
                ("host_admit_s", ctypes.c_double), ("host_launch_s", ctypes.c_double),
                ("host_harvest_s", ctypes.c_double)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p,
                             ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_lock = threading.Lock()
_torch_hooks = None
_D = ctypes.POINTER(ctypes.c_double)


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libibm.so (building it first if asked and absent).  Raises when
    the library is unavailable: there is no CPU fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"{path} is missing: build it with paper_1803_09380_gb300.build")
            _build.build()
        lib = ctypes.CDLL(path)
        vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        lib.ibm_create_lattice.argtypes = [ctypes.POINTER(LatticeDesc), ctypes.POINTER(vp)]
        lib.ibm_add_markers.argtypes = [vp, _D, _D, ci, ctypes.POINTER(BodyDesc), ctypes.POINTER(ci)]
        lib.ibm_step.argtypes = [vp, ci, ctypes.c_uint]
        lib.ibm_read_fields.argtypes = [vp, ci, _D, ctypes.c_size_t]
        lib.ibm_write_fields.argtypes = [vp, ci, _D, ctypes.c_size_t]
        lib.ibm_sync.argtypes = [vp]
        lib.ibm_kernel_times.argtypes = [vp, _D, ctypes.POINTER(ci)]
        lib.ibm_get_sizes.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ci),
                                      ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(ci)]
        lib.ibm_get_counters.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.POINTER(ctypes.c_longlong)]
        lib.ibm_destroy.argtypes = [vp]
        lib.ibm_last_error.argtypes = [vp]
        lib.ibm_last_error.restype = ctypes.c_char_p
        lib.ibm_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, vp]
        lib.ibm_abi_version.restype = ci
        lib.ibm_ib_correct_noalloc.argtypes = [ci, ci, ci, vp, ci, vp, vp, vp, ci, vp, vp, vp]
        lib.ibm_set_option.argtypes = [vp, ci, ctypes.c_longlong]
        lib.ibm_set_marker_velocities.argtypes = [vp, _D, ci]
        lib.ibm_autotune_ib.argtypes = [vp, ctypes.POINTER(ci), ci, ci, ctypes.POINTER(ci), _D]
        lib.ibm_server_create.argtypes = [ctypes.POINTER(ServerDesc), ctypes.POINTER(vp)]
        lib.ibm_server_submit.argtypes = [vp, ctypes.POINTER(CaseDesc), ctypes.POINTER(ctypes.c_longlong)]
        lib.ibm_server_progress.argtypes = [vp, ctypes.POINTER(ci)]
        lib.ibm_server_wait.argtypes = [vp, ctypes.c_longlong]
        lib.ibm_server_result.argtypes = [vp, ctypes.c_longlong, ci, _D, ctypes.c_size_t]
        lib.ibm_server_release.argtypes = [vp, ctypes.c_longlong]
        lib.ibm_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        lib.ibm_server_destroy.argtypes = [vp]
        lib.ibm_server_last_error.argtypes = [vp]
        lib.ibm_server_autotune.argtypes = [vp, ctypes.POINTER(CaseDesc), ci, ctypes.POINTER(ci), ci,
                                            ctypes.POINTER(ci), ci, ctypes.POINTER(ci), ctypes.POINTER(ci),
                                            ctypes.POINTER(ci), _D]
        lib.ibm_server_last_error.restype = ctypes.c_char_p
        for name in SYMBOLS:
            if name not in ("ibm_last_error", "ibm_abi_version", "ibm_server_last_error"):
                getattr(lib, name).restype = ci
        _lib = lib
        return lib


def _check(st: int, h, where: str, allow_warn: bool = False) -> int:
    if st == IBM_OK or (allow_warn and st == IBM_WARN_NOT_CONVERGED):
        return st
    msg = load().ibm_last_error(h).decode(errors="replace")
    raise IBMError(st, where, msg)


def ibm_set_allocator(alloc, release, ctx=None):
    """Install alloc(bytes, device, stream, ctx) / release(ptr, device,
    stream, ctx) as the library's device allocator (None, None: cudaMalloc)."""
    lib = load()
    if alloc is None:
        return _check(lib.ibm_set_allocator(_ALLOC_FN(), _FREE_FN(), None), None, "ibm_set_allocator")
    return _check(lib.ibm_set_allocator(alloc, release, ctx), None, "ibm_set_allocator")


def use_torch_allocator() -> bool:
    """Route the library's device allocations through PyTorch's caching
    allocator.  Returns False when PyTorch CUDA is unavailable."""
    global _torch_hooks
    try:
        import torch
    except ImportError:
        return False
    if not torch.cuda.is_available():
        return False
    if _torch_hooks is not None:
        return True

    def _alloc(nbytes, device, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), int(device), stream or 0))
        except Exception:
            return None

    def _free(ptr, device, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    hooks = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    ibm_set_allocator(hooks[0], hooks[1])
    _torch_hooks = hooks
    return True


def ibm_create_lattice(nx, ny, tau, rho0=1.0, prec="fp32", bc=(PERIODIC,) * 4, wall_u=None,
                       inlet_u=(0.0, 0.0), n_corr=10, corr_tol=0.0, stream=None, device=0,
                       mrt=None, delta_points=4):
    """Create a lattice in the rest equilibrium; returns an opaque handle.
    ``mrt``: None for BGK, else the rates (s_e, s_eps, s_q) of Eq. 6 (a 0
    entry takes the value of section 3)."""
    lib = load()
    d = _lattice_desc(nx, ny, tau, rho0, prec, bc, wall_u, inlet_u, n_corr, corr_tol, mrt, delta_points)
    d.cuda_stream = stream
    d.device = int(device)
    h = ctypes.c_void_p()
    st = lib.ibm_create_lattice(ctypes.byref(d), ctypes.byref(h))
    _check(st, None, "ibm_create_lattice")
    return h


def ibm_add_markers(h, xy, ds=None, kind=BODY_FIXED, xc=(0.0, 0.0), u=(0.0, 0.0), omega=0.0,
                    theta=0.0, rho_s=1.0, rho_f=1.0, volume=0.0, inertia=0.0, radius=0.0,
                    gravity=(0.0, 0.0)) -> int:
    lib = load()
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
    n = xy.shape[0]
    dsp = None
    if ds is not None:
        ds = np.ascontiguousarray(np.broadcast_to(ds, (n,)), dtype=np.float64)
        dsp = ds.ctypes.data_as(_D)
    b = BodyDesc()
    b.kind = int(kind)
    b.xc[0], b.xc[1] = float(xc[0]), float(xc[1])
    b.u[0], b.u[1] = float(u[0]), float(u[1])
    b.omega, b.theta = float(omega), float(theta)
    b.rho_s, b.rho_f, b.volume, b.inertia = float(rho_s), float(rho_f), float(volume), float(inertia)
    b.radius = float(radius)
    b.gravity[0], b.gravity[1] = float(gravity[0]), float(gravity[1])
    bid = ctypes.c_int(-1)
    _check(lib.ibm_add_markers(h, xy.ctypes.data_as(_D), dsp, n, ctypes.byref(b), ctypes.byref(bid)),
           h, "ibm_add_markers")
    return bid.value


def ibm_step(h, nsteps: int, flags: int = STEP_DEFAULT) -> None:
    _check(load().ibm_step(h, int(nsteps), int(flags)), h, "ibm_step")


def ibm_get_sizes(h):
    """(nodes, markers, bodies, band_nodes, band_segments)."""
    n, m, b, bn, bs = (ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(),
                       ctypes.c_int())
    _check(load().ibm_get_sizes(h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(b),
                                ctypes.byref(bn), ctypes.byref(bs)), h, "ibm_get_sizes")
    return n.value, m.value, b.value, bn.value, bs.value


def _field_shape(h, field, nx, ny, n_corr):
    if field in (FIELD_RHO, FIELD_UX, FIELD_UY):
        return (ny, nx)
    if field == FIELD_F:
        return (9, ny, nx)
    if field == FIELD_RESIDUAL:
        return (n_corr + 1,)
    _, m, b, _, _ = ibm_get_sizes(h)
    if field in (FIELD_BODIES, FIELD_BODY_STATE):
        return (b, 9)
    if field == FIELD_MARKERS:
        return (m, 2)
    raise ValueError(f"unknown field {field}")


def ibm_read_fields(h, field: int, nx: int, ny: int, n_corr: int = 0, out=None):
    """Copy a field to a new (or the given) FP64 host array.  Returns
    (array, status); status is IBM_WARN_NOT_CONVERGED for a residual above
    corr_tol, otherwise IBM_OK."""
    shape = _field_shape(h, field, nx, ny, n_corr)
    if out is None:
        out = np.empty(shape, dtype=np.float64)
    assert out.dtype == np.float64 and out.flags.c_contiguous and out.shape == shape
    st = load().ibm_read_fields(h, int(field), out.ctypes.data_as(_D), out.size)
    st = _check(st, h, "ibm_read_fields", allow_warn=True)
    return out, st


def ibm_write_fields(h, field: int, src) -> None:
    src = np.ascontiguousarray(src, dtype=np.float64)
    _check(load().ibm_write_fields(h, int(field), src.ctypes.data_as(_D), src.size), h, "ibm_write_fields")


def ibm_sync(h) -> None:
    _check(load().ibm_sync(h), h, "ibm_sync")


def ibm_kernel_times(h):
    """(total ms, launches) of the collide+stream launches timed since the
    last call."""
    ms, n = ctypes.c_double(), ctypes.c_int()
    _check(load().ibm_kernel_times(h, ctypes.byref(ms), ctypes.byref(n)), h, "ibm_kernel_times")
    return ms.value, n.value


def ibm_get_counters(h):
    """(kernel launches, steps) since creation."""
    k, s = ctypes.c_longlong(), ctypes.c_longlong()
    _check(load().ibm_get_counters(h, ctypes.byref(k), ctypes.byref(s)), h, "ibm_get_counters")
    return k.value, s.value


def ibm_destroy(h) -> None:
    if h is not None and h.value:
        _check(load().ibm_destroy(h), None, "ibm_destroy")
        h.value = None


def ibm_ib_correct_noalloc(nx, ny, prec, f_ptr, n_markers, xy_ptr, ds_ptr, uvel_ptr, n_corr,
                           resid_ptr=None, force_ptr=None, stream=None) -> None:
    """The correction loop on caller-owned device buffers, with no device
    allocation (pointers are raw device addresses; see include/ibm.h)."""
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    _check(load().ibm_ib_correct_noalloc(int(nx), int(ny), p, f_ptr, int(n_markers), xy_ptr, ds_ptr,
                                         uvel_ptr, int(n_corr), resid_ptr, force_ptr, stream),
           None, "ibm_ib_correct_noalloc")


def ibm_set_marker_velocities(h, uv) -> None:
    """Prescribed velocity of every marker of a fixed body, (M, 2) array."""
    uv = np.ascontiguousarray(uv, dtype=np.float64).reshape(-1, 2)
    _check(load().ibm_set_marker_velocities(h, uv.ctypes.data_as(_D), uv.shape[0]), h,
           "ibm_set_marker_velocities")


def ibm_autotune_ib(h, candidates=None, steps_each=20):
    """Measured choice of the correction kernel's CTA count (the candidate
    runs are real steps); returns (best count, microseconds per step)."""
    cand = list(candidates or [])
    arr = (ctypes.c_int * max(len(cand), 1))(*cand)
    best = ctypes.c_int()
    us = ctypes.c_double()
    _check(load().ibm_autotune_ib(h, arr, len(cand), int(steps_each), ctypes.byref(best), ctypes.byref(us)),
           h, "ibm_autotune_ib")
    return best.value, us.value


def ibm_set_option(h, option: int, value: int) -> None:
    _check(load().ibm_set_option(h, int(option), int(value)), h, "ibm_set_option")


def _scheck(st: int, srv, where: str) -> int:
    if st == IBM_OK:
        return st
    msg = load().ibm_server_last_error(srv).decode(errors="replace")
    raise IBMError(st, where, msg)


def ibm_server_create(device=0, max_device_bytes=0.0, max_active=32, steps_per_launch=16,
                      ib_cta_budget=0, ib_markers_per_cta=0, batched=False, tile_nodes=0, corr_first=0):
    d = ServerDesc(int(device), float(max_device_bytes), int(max_active), int(steps_per_launch),
                   int(ib_cta_budget), int(ib_markers_per_cta), int(bool(batched)), int(tile_nodes),
                   int(corr_first))
    srv = ctypes.c_void_p()
    _scheck(load().ibm_server_create(ctypes.byref(d), ctypes.byref(srv)), None, "ibm_server_create")
    return srv


def _lattice_desc(nx, ny, tau, rho0, prec, bc, wall_u, inlet_u, n_corr, corr_tol=0.0, mrt=None,
                  delta_points=4):
    d = LatticeDesc()
    d.nx, d.ny, d.tau, d.rho0 = int(nx), int(ny), float(tau), float(rho0)
    d.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    for k in range(4):
        d.bc[k] = int(bc[k])
    wu = np.zeros(8) if wall_u is None else np.asarray(wall_u, dtype=np.float64).reshape(8)
    for k in range(4):
        d.wall_u[k][0], d.wall_u[k][1] = float(wu[2 * k]), float(wu[2 * k + 1])
    d.inlet_u[0], d.inlet_u[1] = float(inlet_u[0]), float(inlet_u[1])
    d.n_corr, d.corr_tol, d.delta_points = int(n_corr), float(corr_tol), int(delta_points)
    if mrt is not None:
        d.collision = COLL_MRT
        for k in range(3):
            d.mrt_s[k] = float(mrt[k])
    return d


def _body_desc(b) -> BodyDesc:
    bd = BodyDesc()
    bd.kind = int(b.kind)
    bd.xc[0], bd.xc[1] = float(b.xc[0]), float(b.xc[1])
    bd.u[0], bd.u[1] = float(b.u[0]), float(b.u[1])
    bd.omega, bd.theta = float(b.omega), float(b.theta)
    bd.rho_s, bd.rho_f, bd.volume = float(b.rho_s), float(b.rho_f), float(b.volume)
    bd.inertia, bd.radius = float(b.inertia), float(b.radius)
    bd.gravity[0], bd.gravity[1] = float(b.gravity[0]), float(b.gravity[1])
    return bd


def _case_desc_of(case, nsteps, prec, outputs):
    """A CaseDesc for a workloads.Case and the arrays it points to (keep them
    alive while the descriptor is used)."""
    c = CaseDesc()
    c.lattice = _lattice_desc(case.nx, case.ny, case.tau, case.rho0, prec, case.bc, case.wall_u,
                              case.inlet_u, case.n_corr, mrt=case.mrt, delta_points=case.delta_points)
    nb = len(case.bodies)
    bodies = (BodyDesc * max(nb, 1))(*[_body_desc(b) for b in case.bodies])
    nmark = (ctypes.c_int * max(nb, 1))(*[b.xy.shape[0] for b in case.bodies])
    xy = np.ascontiguousarray(np.concatenate([b.xy for b in case.bodies]) if nb else np.zeros((0, 2)))
    ds = np.ascontiguousarray(np.concatenate([b.ds for b in case.bodies]) if nb else np.zeros(0))
    c.nbodies = nb
    c.bodies = bodies
    c.nmarkers = nmark
    c.xy = xy.ctypes.data_as(_D)
    c.ds = ds.ctypes.data_as(_D)
    c.nsteps = int(nsteps)
    c.outputs = int(outputs)
    return c, (bodies, nmark, xy, ds)


def ibm_server_submit(srv, case, nsteps, prec="fp32", outputs=OUT_MACRO | OUT_BODIES | OUT_RESIDUAL) -> int:
    """Submit a workloads.Case for nsteps time steps; returns its id."""
    c, keep = _case_desc_of(case, nsteps, prec, outputs)
    cid = ctypes.c_longlong()
    _scheck(load().ibm_server_submit(srv, ctypes.byref(c), ctypes.byref(cid)), srv, "ibm_server_submit")
    del keep
    return cid.value


def ibm_server_autotune(srv, cases, nsteps, prec="fp32", tile_nodes=None, markers_per_cta=None):
    """Batched mode's autotuner on sample cases (workloads.Case), each run for
    nsteps steps; returns (tile_nodes, markers_per_cta, corr_first, seconds)."""
    descs, keep = [], []
    for case in cases:
        c, k = _case_desc_of(case, nsteps, prec, OUT_RESIDUAL)
        descs.append(c)
        keep.append(k)
    arr = (CaseDesc * len(descs))(*descs)
    tl = list(tile_nodes or [])
    ml = list(markers_per_cta or [])
    ta = (ctypes.c_int * max(len(tl), 1))(*tl)
    ma = (ctypes.c_int * max(len(ml), 1))(*ml)
    bt, bm, bo, sec = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _scheck(load().ibm_server_autotune(srv, arr, len(descs), ta, len(tl), ma, len(ml), ctypes.byref(bt),
                                       ctypes.byref(bm), ctypes.byref(bo), ctypes.byref(sec)),
            srv, "ibm_server_autotune")
    return bt.value, bm.value, bo.value, sec.value


def ibm_server_progress(srv) -> int:
    n = ctypes.c_int()
    _scheck(load().ibm_server_progress(srv, ctypes.byref(n)), srv, "ibm_server_progress")
    return n.value


def ibm_server_wait(srv, case_id=-1) -> None:
    _scheck(load().ibm_server_wait(srv, int(case_id)), srv, "ibm_server_wait")


def ibm_server_result(srv, case_id, field, shape):
    out = np.empty(shape, dtype=np.float64)
    _scheck(load().ibm_server_result(srv, int(case_id), int(field), out.ctypes.data_as(_D), out.size),
            srv, "ibm_server_result")
    return out


def ibm_server_release(srv, case_id) -> None:
    _scheck(load().ibm_server_release(srv, int(case_id)), srv, "ibm_server_release")


def ibm_server_get_stats(srv) -> dict:
    st = ServerStats()
    _scheck(load().ibm_server_get_stats(srv, ctypes.byref(st)), srv, "ibm_server_get_stats")
    return {name: getattr(st, name) for name, _ in ServerStats._fields_}


def ibm_server_destroy(srv) -> None:
    if srv is not None and srv.value:
        load().ibm_server_destroy(srv)
        srv.value = None


def ibm_server_last_error(srv=None) -> str:
    return load().ibm_server_last_error(srv).decode(errors="replace")


class Server:
    """Owning wrapper of an ibm_server (context manager)."""

    def __init__(self, device=0, max_device_bytes=0.0, max_active=32, steps_per_launch=16,
                 ib_cta_budget=0, ib_markers_per_cta=0, batched=False, tile_nodes=0, corr_first=0):
        self.s = ibm_server_create(device, max_device_bytes, max_active, steps_per_launch, ib_cta_budget,
                                   ib_markers_per_cta, batched, tile_nodes, corr_first)
        self._shapes = {}

    def autotune(self, cases, nsteps, prec="fp32", tile_nodes=None, markers_per_cta=None):
        """Batched mode: time the candidate settings on sample cases and keep
        the fastest; returns (tile_nodes, markers_per_cta, corr_first, s)."""
        return ibm_server_autotune(self.s, cases, nsteps, prec, tile_nodes, markers_per_cta)

    def submit(self, case, nsteps, prec="fp32", outputs=OUT_MACRO | OUT_BODIES | OUT_RESIDUAL) -> int:
        cid = ibm_server_submit(self.s, case, nsteps, prec, outputs)
        self._shapes[cid] = (case.ny, case.nx, len(case.bodies), case.n_corr)
        return cid

    def progress(self) -> int:
        return ibm_server_progress(self.s)

    def wait(self, case_id=-1):
        ibm_server_wait(self.s, case_id)

    def result(self, case_id, field):
        ny, nx, nb, nc = self._shapes[case_id]
        shape = {FIELD_RHO: (ny, nx), FIELD_UX: (ny, nx), FIELD_UY: (ny, nx),
                 FIELD_BODIES: (nb, 9), FIELD_RESIDUAL: (nc + 1,)}[field]
        return ibm_server_result(self.s, case_id, field, shape)

    def release(self, case_id):
        ibm_server_release(self.s, case_id)

    def stats(self) -> dict:
        return ibm_server_get_stats(self.s)

    def close(self):
        if getattr(self, "s", None) is not None and self.s.value:
            ibm_server_destroy(self.s)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ibm_last_error(h=None) -> str:
    return load().ibm_last_error(h).decode(errors="replace")


class Lattice:
    """Owning wrapper of one handle (context manager).  Uses a PyTorch
    stream and PyTorch's caching allocator when PyTorch CUDA is present."""

    def __init__(self, nx, ny, tau, rho0=1.0, prec="fp32", bc=(PERIODIC,) * 4, wall_u=None,
                 inlet_u=(0.0, 0.0), n_corr=10, corr_tol=0.0, device=0, torch_stream=True,
                 mrt=None, delta_points=4):
        self.nx, self.ny, self.n_corr = int(nx), int(ny), int(n_corr)
        self.prec = prec
        self._stream = None
        stream_ptr = None
        if torch_stream:
            try:
                import torch
                if torch.cuda.is_available():
                    use_torch_allocator()
                    self._stream = torch.cuda.Stream(device=device)
                    stream_ptr = self._stream.cuda_stream
            except ImportError:
                pass
        self.h = ibm_create_lattice(nx, ny, tau, rho0, prec, bc, wall_u, inlet_u, n_corr,
                                    corr_tol, stream_ptr, device, mrt, delta_points)

    @classmethod
    def from_case(cls, case, prec="fp32", **kw):
        kw.setdefault("mrt", case.mrt)
        kw.setdefault("delta_points", case.delta_points)
        lat = cls(case.nx, case.ny, case.tau, case.rho0, prec, case.bc, case.wall_u, case.inlet_u,
                  case.n_corr, **kw)
        for b in case.bodies:
            lat.add_markers(b.xy, b.ds, **b.as_kwargs())
        return lat

    def add_markers(self, xy, ds=None, **body) -> int:
        return ibm_add_markers(self.h, xy, ds, **body)

    def step(self, n=1, flags=STEP_DEFAULT):
        ibm_step(self.h, n, flags)

    def read(self, field, out=None):
        return ibm_read_fields(self.h, field, self.nx, self.ny, self.n_corr, out)[0]

    def write(self, field, src):
        ibm_write_fields(self.h, field, src)

    def moments(self):
        return self.read(FIELD_RHO), self.read(FIELD_UX), self.read(FIELD_UY)

    @property
    def f(self):
        return self.read(FIELD_F)

    @f.setter
    def f(self, value):
        self.write(FIELD_F, value)

    @property
    def resid(self):
        return self.read(FIELD_RESIDUAL)

    @property
    def bodies(self):
        return self.read(FIELD_BODIES)

    @property
    def markers(self):
        return self.read(FIELD_MARKERS)

    def checkpoint(self) -> dict:
        """Everything a lattice made with the same parameters and bodies needs
        to continue this run bit for bit: the populations and the bodies'
        pose and velocities (current and previous step)."""
        return {"f": self.read(FIELD_F), "body_state": self.read(FIELD_BODY_STATE)}

    def restore(self, state: dict) -> None:
        self.write(FIELD_F, state["f"])
        self.write(FIELD_BODY_STATE, state["body_state"])

    def init_equilibrium(self, rho, ux, uy):
        shp = (self.ny, self.nx)
        a = np.stack([np.broadcast_to(rho, shp), np.broadcast_to(ux, shp), np.broadcast_to(uy, shp)])
        self.write(FIELD_MACRO_INIT, a)

    def sync(self):
        ibm_sync(self.h)

    def sizes(self):
        return ibm_get_sizes(self.h)

    def kernel_times(self):
        return ibm_kernel_times(self.h)

    def set_marker_velocities(self, uv) -> None:
        """Prescribed U_l of every marker of a fixed body from the next step on."""
        ibm_set_marker_velocities(self.h, uv)

    def set_ib_ctas(self, n: int) -> None:
        """CTAs of the correction-loop kernel (0: the default choice)."""
        ibm_set_option(self.h, IBM_OPT_IB_CTAS, n)

    def autotune_ib(self, candidates=None, steps_each=20):
        """Pick the correction kernel's CTA count by timing candidates (the
        candidate runs advance the simulation); returns (count, us/step)."""
        return ibm_autotune_ib(self.h, candidates, steps_each)

    def set_ib_threads(self, n: int) -> None:
        """Threads per correction-loop CTA: 256, 512 or 1024."""
        ibm_set_option(self.h, IBM_OPT_IB_THREADS, n)

    def counters(self):
        return ibm_get_counters(self.h)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            ibm_destroy(self.h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
