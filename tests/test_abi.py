"""The C ABI library builds for sm_103a, loads, and exports every entry point that include/nmgb.h
declares.  No GPU needed: only host-side argument validation and size arithmetic are called."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(nm_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_2411_11725_gb300 as nmgb
    return nmgb.load()


def test_every_declared_symbol_is_exported(lib):
    import paper_2411_11725_gb300 as nmgb
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    bound = {s[0] for s in nmgb.SIGNATURES}
    assert set(declared) <= bound, set(declared) - bound


def test_library_is_sm103a_build():
    import paper_2411_11725_gb300 as nmgb
    assert "arch=compute_103a,code=sm_103a" in nmgb._build.ARCH
    assert os.path.exists(nmgb.lib_path())


def test_host_side_validation(lib):
    h = ctypes.c_void_p()
    assert lib.nm_create_mesh(0, 4, 4, 1e-9, 1e-9, 1e-9, 0, None, ctypes.byref(h)) == -1
    assert b"cell counts" in lib.nm_last_error()
    assert lib.nm_create_mesh(4, 4, 4, -1e-9, 1e-9, 1e-9, 0, None, ctypes.byref(h)) == -1
    assert lib.nm_create_mesh(4, 4, 4, 1e-9, 1e-9, 1e-9, 7, None, ctypes.byref(h)) == -1
    assert lib.nm_create_mesh(4, 4, 4, 1e-9, 1e-9, 1e-9, 0, None, None) == -1
    assert lib.nm_create_mesh(4096, 4, 4, 1e-9, 1e-9, 1e-9, 0, None, ctypes.byref(h)) == -1
    for basis in (0, 4):
        assert lib.nm_create_mesh_basis(4, 4, 4, 1e-9, 1e-9, 1e-9, 0, basis, None, ctypes.byref(h)) == -1
        assert b"basis must be" in lib.nm_last_error()
    assert lib.nm_create_mesh_basis(0, 1, 1, 1e-9, 1e-9, 1e-9, 0, 1, None, ctypes.byref(h)) == -1
    assert lib.nm_destroy_mesh(None) == 0
    assert lib.nm_set_terms(None, 1) == -1
    assert lib.nm_sync(None) == -1


def test_footprint_arithmetic(lib):
    small = lib.nm_footprint_bytes(16, 16, 4, 0)
    big = lib.nm_footprint_bytes(1024, 1024, 32, 0)
    f64 = lib.nm_footprint_bytes(1024, 1024, 32, 1)
    assert 0 < small < big < f64
    # the largest throughput grid fits comfortably in one GB300's HBM
    assert big < 20e9 and f64 < 40e9
    assert lib.nm_footprint_bytes(0, 1, 1, 0) == -1


def _request(nmgb, **kw):
    import numpy as np
    n = kw.pop("n", (8, 8, 2))
    m0 = np.zeros((n[0] + 1, n[1] + 1, n[2] + 1, 3))
    m0[..., 2] = 1
    r = nmgb.Request()
    r.n = (ctypes.c_int * 3)(*n)
    r.dx = (ctypes.c_double * 3)(*kw.pop("dx", (3e-9, 3e-9, 3e-9)))
    r.precision = kw.pop("precision", 0)
    r.Ms, r.A, r.Ku = kw.pop("Ms", 8e5), 1.3e-11, 0.0
    r.axis = (ctypes.c_double * 3)(0, 0, 1)
    r.alpha, r.gamma = 0.1, 2.2e5
    r.terms = kw.pop("terms", 13)
    r.method = kw.pop("method", 2)
    r.t_end = kw.pop("t_end", 1e-12)
    r.rtol = r.atol = kw.pop("tol", 1e-5)
    r.dt0 = kw.pop("dt0", 1e-14)
    r.m0 = None if kw.pop("no_m0", False) else m0.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return r, m0


def test_server_host_side_validation(lib):
    """Request and server arguments are checked on the host before any CUDA call."""
    import paper_2411_11725_gb300 as nmgb
    h = ctypes.c_void_p()
    assert lib.nm_server_create(0, 4, ctypes.byref(h)) == -1
    assert lib.nm_server_create(1 << 30, 0, ctypes.byref(h)) == -1
    assert lib.nm_server_create(1 << 30, 4, None) == -1
    assert lib.nm_server_destroy(None) == 0
    cases = [dict(n=(0, 8, 1)), dict(n=(2048, 8, 1)), dict(dx=(0, 1e-9, 1e-9)), dict(precision=3),
             dict(Ms=-1.0), dict(terms=64), dict(method=7), dict(t_end=0.0), dict(dt0=-1.0), dict(tol=0.0),
             dict(no_m0=True)]
    for kw in cases:
        r, _ = _request(nmgb, **kw)
        assert lib.nm_server_submit(None, ctypes.byref(r)) == -1, kw
        assert b"server is NULL" not in lib.nm_last_error(), kw
    r, _ = _request(nmgb)
    assert lib.nm_server_submit(None, ctypes.byref(r)) == -1
    assert b"server is NULL" in lib.nm_last_error()
    n = ctypes.c_int()
    assert lib.nm_server_poll(None, None, 0, 0.0, ctypes.byref(n)) == -1
