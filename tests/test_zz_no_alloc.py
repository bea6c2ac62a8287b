"""nm_get_state_noalloc (read-back of the state through a fixed device staging array, no allocation)
against nm_get_state, called through the C ABI on two calls in a row with a state change between them;
meshes beyond the array's size are refused; and the calls allocate no device memory: neither the
high-water mark of the device's default memory pool (where stream-ordered allocations come from) nor
the device's free memory moves, while nm_get_state moves the former."""
import ctypes

import numpy as np
import pytest

import nm_inputs as inp
from helpers import gpu_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nmgb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_11725_gb300 as nmgb
    nmgb.load()
    return nmgb


def _cudart():
    # the CUDA runtime the library is linked against is already loaded in this process
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    raise RuntimeError("CUDA runtime library not found")


_USED_MEM_HIGH = 8  # cudaMemPoolAttrUsedMemHigh


def _pool_high(rt, pool):
    v = ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, _USED_MEM_HIGH, ctypes.byref(v)) == 0
    return v.value


def _pool_reset_high(rt, pool):
    zero = ctypes.c_uint64(0)
    assert rt.cudaMemPoolSetAttribute(pool, _USED_MEM_HIGH, ctypes.byref(zero)) == 0


def _free_bytes(rt):
    free, total = ctypes.c_size_t(), ctypes.c_size_t()
    assert rt.cudaMemGetInfo(ctypes.byref(free), ctypes.byref(total)) == 0
    return free.value


def _noalloc(lib, me, out):
    t, dt = ctypes.c_double(), ctypes.c_double()
    rc = lib.nm_get_state_noalloc(me._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(t),
                                  ctypes.byref(dt))
    return rc, t.value, dt.value


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_read_back_equals_get_state(nmgb, precision):
    lib = nmgb.load()
    p = inp.random_problem(np.random.default_rng(60), (12, 9, 4), vacuum=True)
    me = gpu_mesh(nmgb, p, precision)
    me.set_state(p.m0, 0.0, 1e-14)
    for call in range(2):
        out = np.full(p.nodes + (3,), np.nan)
        rc, t, dt = _noalloc(lib, me, out)
        assert rc == 0, lib.nm_last_error()
        ref, t_ref, dt_ref = me.get_state()
        assert np.array_equal(out, ref) and t == t_ref and dt == dt_ref
        if call == 0:
            assert np.array_equal(out, p.m0)
            me.run_steps(3, nmgb.DP54, 1e-5, 1e-5)
    assert t > 0 and not np.array_equal(out, p.m0)
    me.close()


def test_noalloc_refuses_meshes_beyond_the_array(nmgb):
    lib = nmgb.load()
    me = nmgb.Mesh((64, 64, 64), (3e-9,) * 3, nmgb.F32)  # 65^3 = 274625 nodes > 174762
    out = np.zeros((65, 65, 65, 3))
    rc, _, _ = _noalloc(lib, me, out)
    assert rc == nmgb.ERR_ARG and b"at most 174762" in lib.nm_last_error()
    me.close()


def test_noalloc_allocates_no_device_memory(nmgb):
    import torch
    lib = nmgb.load()
    rt = _cudart()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    p = inp.random_problem(np.random.default_rng(61), (12, 9, 4), vacuum=False)
    me = gpu_mesh(nmgb, p, 0)
    me.set_state(p.m0, 0.0, 1e-14)
    out = np.zeros(p.nodes + (3,))
    assert _noalloc(lib, me, out)[0] == 0  # first call on the device: looks up the array's address
    torch.cuda.synchronize()
    # the probe sees stream-ordered allocations: nm_get_state stages its copy in one
    _pool_reset_high(rt, pool)
    me.get_state()
    assert _pool_high(rt, pool) >= out.nbytes
    _pool_reset_high(rt, pool)
    free0 = _free_bytes(rt)
    for _ in range(2):
        rc, _, _ = _noalloc(lib, me, out)
        assert rc == 0, lib.nm_last_error()
    assert _pool_high(rt, pool) == 0
    assert _free_bytes(rt) == free0
    assert np.array_equal(out, me.get_state()[0])
    me.close()


def test_noalloc_clears_an_earlier_error_message(nmgb):
    lib = nmgb.load()
    big = nmgb.Mesh((64, 64, 64), (3e-9,) * 3, nmgb.F32)
    assert _noalloc(lib, big, np.zeros((65, 65, 65, 3)))[0] == nmgb.ERR_ARG
    assert lib.nm_last_error() != b""
    p = inp.random_problem(np.random.default_rng(62), (4, 3, 2))
    me = gpu_mesh(nmgb, p, 1)
    me.set_state(p.m0, 0.0, 1e-14)
    assert _noalloc(lib, me, np.zeros(p.nodes + (3,)))[0] == 0
    assert lib.nm_last_error() == b""
    me.close()
    big.close()
