"""Parity of the GPU effective field (all terms, FP64 and FP32 paths) with the FP64 oracle.

Tolerances (relative L2 over all nodes and components): FP64 path 1e-12, FP32 path 1e-5, with the
oracle fed the same rounded input (FP32 values promoted to FP64) so that only kernel error counts.
"""
import numpy as np
import pytest

import nm_inputs as inp
from helpers import gpu_mesh, oracle_mesh, rel_l2, rounded

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}


@pytest.fixture(scope="module")
def nmgb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_11725_gb300 as nmgb
    nmgb.load()
    return nmgb


def _heff_gpu(nmgb, p, precision, m, terms, t=0.0):
    import torch
    me = gpu_mesh(nmgb, p, precision)
    mt = torch.tensor(m, dtype=me.dtype, device="cuda")
    h = me.h_eff(mt, terms, t).double().cpu().numpy()
    me.close()
    return h


# N3 = 2..64 covers every z transform length (P3 = 4, 8, 16, 32, 64 in registers for FP32, 128 through
# shared memory), full and ragged, up to the largest supported N3
SHAPES = [(1, 1, 1), (2, 1, 1), (3, 2, 1), (5, 3, 2), (7, 1, 3), (4, 6, 1), (13, 7, 5), (16, 16, 4), (9, 11, 3),
          (1, 5, 4), (6, 5, 9), (3, 4, 16), (3, 4, 20), (2, 3, 32), (2, 3, 33), (5, 4, 48), (3, 2, 64),
          (1, 1, 64)]


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("shape", SHAPES)
def test_heff_all_terms_random_material(oracle_mod, nmgb, precision, shape):
    rng = np.random.default_rng(hash(shape) % 1000)
    p = inp.random_problem(rng, shape, vacuum=False)
    m = rounded(p.m0, precision)
    t = 1.7e-10
    ref = oracle_mesh(oracle_mod, p).h_eff(m, oracle_mod.ALL, t)
    h = _heff_gpu(nmgb, p, precision, m, oracle_mod.ALL, t)
    assert rel_l2(h, ref) < TOL[precision]


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("term", ["EXCH", "ANIS", "ZEE", "DEMAG"])
def test_heff_single_terms(oracle_mod, nmgb, precision, term):
    rng = np.random.default_rng(5)
    p = inp.random_problem(rng, (6, 5, 3), vacuum=True)
    m = rounded(p.m0, precision)
    T = getattr(oracle_mod, term)
    ref = oracle_mesh(oracle_mod, p).h_eff(m, T, 0.3e-9)
    h = _heff_gpu(nmgb, p, precision, m, T, 0.3e-9)
    assert rel_l2(h, ref) < TOL[precision], term


@pytest.mark.parametrize("precision", [1, 0])
def test_heff_vacuum_nodes_zero(oracle_mod, nmgb, precision):
    rng = np.random.default_rng(9)
    p = inp.random_problem(rng, (8, 6, 3), vacuum=True)
    Ms = p.Ms_cells()
    Ms[:, :, :] = 0.0
    Ms[2:5, 1:4, 1] = 7e5
    p.Ms = Ms
    m = rounded(p.m0, precision)
    ref = oracle_mesh(oracle_mod, p).h_eff(m, oracle_mod.ALL)
    h = _heff_gpu(nmgb, p, precision, m, oracle_mod.ALL)
    assert rel_l2(h, ref) < TOL[precision]
    assert np.all(h[ref == 0] == 0)


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("which", ["cuboid_rk4", "thin_film", "waveguide"])
def test_heff_workloads(oracle_mod, nmgb, precision, which):
    p = getattr(inp, which)(0)
    m = rounded(p.m0 if which != "waveguide" else inp.unit_vectors(np.random.default_rng(3), p.nodes), precision)
    ref = oracle_mesh(oracle_mod, p).h_eff(m, oracle_mod.ALL, 1.1e-10)
    h = _heff_gpu(nmgb, p, precision, m, oracle_mod.ALL, 1.1e-10)
    assert rel_l2(h, ref) < TOL[precision]


def test_heff_deterministic(oracle_mod, nmgb):
    import torch
    p = inp.cuboid_rk4(1)
    me = gpu_mesh(nmgb, p, 0)
    mt = torch.tensor(p.m0, dtype=torch.float32, device="cuda")
    a = me.h_eff(mt, 15).cpu().numpy()
    b = me.h_eff(mt, 15).cpu().numpy()
    assert np.array_equal(a, b)
