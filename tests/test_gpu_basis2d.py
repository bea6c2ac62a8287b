"""2D nodal basis with full 3D integration on the GPU (nm_create_mesh_basis(..., 2, ...), section
"Low-Dimensional Geometries"): effective field and LLG steps against the oracle's 2D basis (the 3D
Galerkin system restricted to z-constant m), FP64 rel-L2 <= 1e-12 and FP32 <= 1e-5.
"""
import numpy as np
import pytest

import nm_inputs as inp
from helpers import rel_l2, rounded

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


def _m2(rng, p):
    return inp.unit_vectors(rng, (p.n[0] + 1, p.n[1] + 1, 1))


def _oracle2(oracle_mod, p):
    from oracle import basis2d
    me = basis2d.Mesh2D(p.n, p.dx)
    me.set_material(p.Ms_cells(), p.A_cells(), p.Ku_cells(), p.axis, p.alpha, p.gamma)
    me.set_zeeman(p.h_uniform, p.h_freq, p.h_phase, p.h_cell, p.cell_freq, p.cell_phase)
    return me


def _gpu2(nmgb, p, precision):
    me = nmgb.Mesh(p.n, p.dx, precision, basis=2)
    def arg(v):
        return v if np.ndim(v) == 0 else np.asarray(v, dtype=np.float64)
    me.set_material(arg(p.Ms), arg(p.A), arg(p.Ku), p.axis, p.alpha, p.gamma)
    me.set_zeeman(p.h_uniform, p.h_freq, p.h_phase, p.h_cell, p.cell_freq, p.cell_phase)
    me.set_terms(p.terms)
    return me


def _h_gpu(nmgb, me, m, terms, t):
    import torch
    mt = torch.tensor(m, dtype=me.dtype, device="cuda")
    return me.h_eff(mt, terms, t).double().cpu().numpy()


SHAPES = [(1, 1, 1), (3, 2, 1), (7, 5, 1), (13, 7, 2), (9, 11, 3), (16, 16, 1), (5, 1, 4)]


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("vacuum", [False, True])
def test_heff_matches_oracle(oracle_mod, nmgb, precision, shape, vacuum):
    rng = np.random.default_rng(hash((shape, vacuum)) % 1000)
    p = inp.random_problem(rng, shape, vacuum=vacuum)
    m = rounded(_m2(rng, p), precision)
    ref = _oracle2(oracle_mod, p).h_eff(m, oracle_mod.ALL, 2.3e-10)
    me = _gpu2(nmgb, p, precision)
    h = _h_gpu(nmgb, me, m, oracle_mod.ALL, 2.3e-10)
    me.close()
    assert h.shape == ref.shape
    assert rel_l2(h, ref) < TOL[precision]


@pytest.mark.parametrize("term", ["EXCH", "ANIS", "ZEE", "DEMAG"])
def test_single_terms(oracle_mod, nmgb, term):
    rng = np.random.default_rng(5)
    p = inp.random_problem(rng, (12, 9, 2))
    m = _m2(rng, p)
    bit = getattr(oracle_mod, term)
    ref = _oracle2(oracle_mod, p).h_eff(m, bit, 0.7e-10)
    me = _gpu2(nmgb, p, 1)
    h = _h_gpu(nmgb, me, m, bit, 0.7e-10)
    me.close()
    assert rel_l2(h, ref) < 1e-12


def test_rk4_steps_match_oracle(oracle_mod, nmgb):
    rng = np.random.default_rng(6)
    p = inp.random_problem(rng, (10, 7, 2))
    om = _oracle2(oracle_mod, p)
    m = _m2(rng, p)
    steps, dt = 30, 1e-14
    ref = m.copy()
    for s in range(steps):
        ref = om.rk4_step(ref, s * dt, dt, oracle_mod.ALL, renorm=True)
    for prec, tol in ((1, 1e-12), (0, 1e-5)):
        me = _gpu2(nmgb, p, prec)
        me.set_state(m, 0.0, dt)
        me.run_steps(steps, nmgb.RK4, 0.0, 0.0)
        mg, t, _ = me.get_state()
        me.close()
        assert abs(t - steps * dt) <= 1e-12 * steps * dt
        assert rel_l2(mg, ref) < tol


def test_thin_film_dp5_runs_and_halves_the_nodes(nmgb):
    """The thin-film workload on one node layer: adaptive steps run, |m| stays 1, and the 2D mesh holds
    (N1+1)(N2+1) nodes against twice that for the trilinear basis of one cell layer."""
    p = inp.thin_film(0)
    me = _gpu2(nmgb, p, 0)
    m0 = p.m0[:, :, :1, :]
    me.set_state(m0, 0.0, 1e-13)
    me.run_steps(20, nmgb.DP54, 1e-5, 1e-5)
    m, t, _ = me.get_state()
    assert t > 0 and np.abs(np.linalg.norm(m, axis=-1) - 1).max() < 1e-12
    assert me.info()["n_nodes"] * 2 == int(np.prod(p.nodes))
    me.close()


def test_dmi_needs_the_3d_basis(nmgb):
    rng = np.random.default_rng(7)
    p = inp.random_problem(rng, (3, 3, 1))
    me = _gpu2(nmgb, p, 1)
    with pytest.raises(nmgb.NMError):
        me.set_dmi(1e-3)
    me.close()
