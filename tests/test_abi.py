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
