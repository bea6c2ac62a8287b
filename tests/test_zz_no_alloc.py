"""nm_get_state_noalloc (read-back of the state through a fixed device staging array, no allocation)
against nm_get_state, called through the C ABI on two calls in a row with a state change between them;
meshes beyond the array's size are refused."""
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
