"""1D nodal basis with full 3D integration on the GPU (nm_create_mesh_basis(..., 1, ...), section
"Low-Dimensional Geometries"): effective field and LLG steps against the oracle's 1D basis (the 3D
Galerkin system restricted to m that depends on x alone), FP64 rel-L2 <= 1e-12 and FP32 <= 1e-5.
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


def _m1(rng, p):
    return inp.unit_vectors(rng, (p.n[0] + 1, 1, 1))


def _oracle1(p):
    from oracle import basis1d
    me = basis1d.Mesh1D(p.n, p.dx)
    me.set_material(p.Ms_cells(), p.A_cells(), p.Ku_cells(), p.axis, p.alpha, p.gamma)
    me.set_zeeman(p.h_uniform, p.h_freq, p.h_phase, p.h_cell, p.cell_freq, p.cell_phase)
    return me


def _gpu1(nmgb, p, precision):
    me = nmgb.Mesh(p.n, p.dx, precision, basis=1)
    def arg(v):
        return v if np.ndim(v) == 0 else np.asarray(v, dtype=np.float64)
    me.set_material(arg(p.Ms), arg(p.A), arg(p.Ku), p.axis, p.alpha, p.gamma)
    me.set_zeeman(p.h_uniform, p.h_freq, p.h_phase, p.h_cell, p.cell_freq, p.cell_phase)
    me.set_terms(p.terms)
    return me


def _h_gpu(me, m, terms, t):
    import torch
    mt = torch.tensor(m, dtype=me.dtype, device="cuda")
    return me.h_eff(mt, terms, t).double().cpu().numpy()


# single cells, wires of one cell cross-section, small and ragged cross-sections, and one cross-section
# of more cells (144) than a node block has threads (128)
SHAPES = [(1, 1, 1), (2, 1, 1), (7, 1, 1), (13, 3, 2), (9, 4, 3), (30, 2, 2), (5, 1, 4), (12, 16, 9)]


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("vacuum", [False, True])
def test_heff_matches_oracle(oracle_mod, nmgb, precision, shape, vacuum):
    rng = np.random.default_rng(hash((shape, vacuum, 1)) % 1000)
    p = inp.random_problem(rng, shape, vacuum=vacuum)
    m = rounded(_m1(rng, p), precision)
    ref = _oracle1(p).h_eff(m, oracle_mod.ALL, 2.3e-10)
    me = _gpu1(nmgb, p, precision)
    h = _h_gpu(me, m, oracle_mod.ALL, 2.3e-10)
    me.close()
    assert h.shape == ref.shape == (shape[0] + 1, 1, 1, 3)
    assert rel_l2(h, ref) < TOL[precision]


@pytest.mark.parametrize("term", ["EXCH", "ANIS", "ZEE", "DEMAG"])
def test_single_terms(oracle_mod, nmgb, term):
    rng = np.random.default_rng(15)
    p = inp.random_problem(rng, (20, 3, 2))
    m = _m1(rng, p)
    bit = getattr(oracle_mod, term)
    ref = _oracle1(p).h_eff(m, bit, 0.7e-10)
    me = _gpu1(nmgb, p, 1)
    h = _h_gpu(me, m, bit, 0.7e-10)
    me.close()
    assert rel_l2(h, ref) < 1e-12


def test_rk4_steps_match_oracle(oracle_mod, nmgb):
    rng = np.random.default_rng(16)
    p = inp.random_problem(rng, (24, 2, 3), vacuum=True)
    om = _oracle1(p)
    m = _m1(rng, p)
    steps, dt = 30, 1e-14
    ref = m.copy()
    for s in range(steps):
        ref = om.rk4_step(ref, s * dt, dt, oracle_mod.ALL, renorm=True)
    for prec, tol in ((1, 1e-12), (0, 1e-5)):
        me = _gpu1(nmgb, p, prec)
        me.set_state(m, 0.0, dt)
        me.run_steps(steps, nmgb.RK4, 0.0, 0.0)
        mg, t, _ = me.get_state()
        me.close()
        assert abs(t - steps * dt) <= 1e-12 * steps * dt
        assert rel_l2(mg, ref) < tol


def test_wire_dp5_runs_on_one_node_row(nmgb):
    """Adaptive steps on a 256-cell wire of 2 x 2 cells: the mesh holds N1 + 1 nodes, the steps run and
    |m| stays 1."""
    rng = np.random.default_rng(17)
    p = inp.random_problem(rng, (256, 2, 2))
    me = _gpu1(nmgb, p, 0)
    me.set_state(_m1(rng, p), 0.0, 1e-14)
    me.run_steps(20, nmgb.DP54, 1e-5, 1e-5)
    m, t, _ = me.get_state()
    assert t > 0 and np.abs(np.linalg.norm(m, axis=-1) - 1).max() < 1e-12
    assert me.info()["n_nodes"] == 257
    me.close()


def test_dmi_needs_the_3d_basis(nmgb):
    rng = np.random.default_rng(18)
    p = inp.random_problem(rng, (4, 2, 1))
    me = _gpu1(nmgb, p, 1)
    with pytest.raises(nmgb.NMError):
        me.set_dmi(1e-3)
    me.close()
