"""Host-side checks of the C ABI: the CUDA library builds for sm_103a, loads,
and exports every entry point include/ibm.h declares; argument checks that
need no GPU; the seeded workload generators."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_1803_09380_gb300 import build as libbuild
from paper_1803_09380_gb300 import ibm
from paper_1803_09380_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ibm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ibm_[a-z_]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    path = libbuild.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert "ibm_step" in syms and "ibm_create_lattice" in syms
    for name in syms:
        assert hasattr(lib, name), f"{name} declared in ibm.h but not exported"
    hdr = open(os.path.join(ROOT, "include", "ibm.h")).read()
    assert lib.ibm_abi_version() == int(re.search(r"#define IBM_ABI_VERSION (\d+)", hdr).group(1))


def test_descriptor_layout_matches_the_header():
    """The ctypes mirror of ibm_lattice_desc ends with the collision fields
    at the offsets a C compiler gives them (natural alignment)."""
    d = ibm.LatticeDesc
    assert d.collision.offset == d.device.offset + 4
    assert d.mrt_s.offset % 8 == 0 and d.mrt_s.offset >= d.collision.offset + 4
    assert ctypes.sizeof(d) == d.mrt_s.offset + 24


def test_binding_covers_every_declared_symbol():
    for name in declared_symbols():
        assert name in ibm.SYMBOLS, f"{name} has no binding"


def test_null_arguments_are_rejected_without_a_gpu():
    lib = ibm.load()
    h = ctypes.c_void_p()
    assert lib.ibm_create_lattice(None, ctypes.byref(h)) == ibm.IBM_ERR_INVALID
    assert "desc is NULL" in ibm.ibm_last_error(None)
    assert lib.ibm_step(None, 1, 0) == ibm.IBM_ERR_INVALID
    assert lib.ibm_destroy(None) == ibm.IBM_OK


@pytest.mark.parametrize("kw,msg", [
    (dict(nx=3), "nx and ny"),
    (dict(tau=0.5), "tau"),
    (dict(tau=float("nan")), "tau"),
    (dict(bc=(0, 1, 0, 0)), "paired"),
    (dict(bc=(1, 3, 1, 1)), "inlet"),
    (dict(bc=(4, 1, 1, 1)), "outlet"),
    (dict(n_corr=-1), "n_corr"),
    (dict(prec=9), "precision"),
])
def test_create_rejects_bad_descriptors_before_touching_the_gpu(kw, msg):
    args = dict(nx=16, ny=16, tau=0.8)
    args.update(kw)
    with pytest.raises(ibm.IBMError) as e:
        ibm.ibm_create_lattice(**args)
    assert e.value.status == ibm.IBM_ERR_INVALID
    assert msg in str(e.value)


def test_ring_markers_spacing_and_arc_length():
    xy, ds = wl.ring(32.0, 32.0, 10.0)
    assert xy.shape == (63, 2)
    r = np.hypot(xy[:, 0] - 32, xy[:, 1] - 32)
    assert np.allclose(r, 10.0)
    assert np.allclose(ds, 2 * math.pi * 10 / 63)
    gaps = np.hypot(*np.diff(np.vstack([xy, xy[:1]]), axis=0).T)
    assert np.all(np.abs(gaps - 1.0) < 0.01)


def test_couette_sweep_marker_counts():
    counts = {64: (63, 157), 128: (125, 314), 512: (502, 1255), 4096: (4015, 10037)}
    for n, (m1, m2) in counts.items():
        c = wl.couette(n)
        assert c.bodies[0].xy.shape[0] == m1 and c.bodies[1].xy.shape[0] == m2


def test_seeded_generators_are_reproducible():
    a = wl.random_perturbation(8, 8, seed=5)
    b = wl.random_perturbation(8, 8, seed=5)
    assert np.array_equal(a, b)
    r1 = wl.random_fields(8, 8, seed=2)
    r2 = wl.random_fields(8, 8, seed=2)
    assert all(np.array_equal(x, y) for x, y in zip(r1, r2))
