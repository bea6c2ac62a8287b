"""Pins of the oracle's sampled evaluation (``oracle.sampled``), which the full-size parity tests use:
on meshes small enough for the whole-mesh oracle, the value at every sampled node equals the whole-mesh
value.  Heterogeneous material, vacuum cells, cell-wise fields and DMI exercise the restriction argument
(cells holding the node), the Runge-Kutta dependence radius and the sparse direct demag sum."""
import numpy as np
import pytest

import nm_inputs as inp


@pytest.fixture(scope="module")
def sampled():
    from oracle import sampled as s
    return s


def _material(p):
    return (p.Ms_cells(), p.A_cells(), p.Ku_cells(), p.axis, p.alpha, p.gamma)


def test_local_field_equals_whole_mesh(oracle_mod, sampled):
    rng = np.random.default_rng(31)
    p = inp.random_problem(rng, (7, 6, 5), vacuum=True)
    D = rng.uniform(-3e-3, 3e-3, p.n)
    zee = dict(h_uniform=p.h_uniform, freq=p.h_freq, phase=p.h_phase, h_cell=p.h_cell, cell_freq=p.cell_freq,
               cell_phase=p.cell_phase)
    me = oracle_mod.Mesh(p.n, p.dx)
    me.set_material(*_material(p))
    me.set_zeeman(**zee)
    me.set_dmi(D)
    terms = oracle_mod.EXCH | oracle_mod.ANIS | oracle_mod.ZEE | oracle_mod.DMI
    t = 0.4e-10
    ref = me.h_eff(p.m0, terms, t)
    for node in np.ndindex(*p.nodes):
        h = sampled.local_field_at(p.n, p.dx, _material(p), p.m0, node, terms, t, zee, D)
        np.testing.assert_allclose(h, ref[node], rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_dp5_step_equals_whole_mesh(oracle_mod, sampled):
    """Nodes deep inside a 20x18x16 mesh and on its faces, edges and corners: the step on the cells
    within 6 nodes reproduces the whole-mesh step."""
    rng = np.random.default_rng(32)
    p = inp.random_problem(rng, (20, 18, 16))
    terms = oracle_mod.EXCH | oracle_mod.ANIS
    dt = 2e-14
    me = oracle_mod.Mesh(p.n, p.dx)
    me.set_material(*_material(p))
    st = me.dp5_stepper(p.m0, 0.0, dt, terms, rtol=1e3, atol=1e3, renorm=True)
    assert st.step()
    ref = st.m
    nodes = [(10, 9, 8), (0, 0, 0), (20, 18, 16), (3, 17, 8), (10, 0, 16), (7, 9, 1), (19, 2, 12)]
    for node in nodes:
        m1 = sampled.dp5_step_at(p.n, p.dx, _material(p), p.m0, node, terms, dt)
        np.testing.assert_allclose(m1, ref[node], rtol=0, atol=1e-13)
    # a cut one node closer changes the deep node (the radius is tight): shown on a five times longer
    # step, where the sixth-order coupling is above rounding
    node, dt5 = (10, 9, 8), 1e-13
    st = me.dp5_stepper(p.m0, 0.0, dt5, terms, rtol=1e3, atol=1e3, renorm=True)
    assert st.step()
    exact = sampled.dp5_step_at(p.n, p.dx, _material(p), p.m0, node, terms, dt5)
    assert np.abs(exact - st.m[node]).max() <= 1e-13
    me_cut, lo, hi, local = sampled.submesh(p.n, p.dx, _material(p), node, 5)
    st_cut = me_cut.dp5_stepper(np.ascontiguousarray(p.m0[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1]),
                                0.0, dt5, terms, rtol=1e3, atol=1e3, renorm=True)
    assert st_cut.step()
    assert np.abs(st_cut.m[local] - st.m[node]).max() > 1e-12


def test_sparse_demag_equals_whole_mesh(oracle_mod, sampled):
    rng = np.random.default_rng(33)
    p = inp.random_problem(rng, (9, 7, 5), vacuum=True)
    m = np.zeros(p.nodes + (3,))
    for node in [(0, 0, 0), (4, 3, 2), (5, 3, 2), (9, 7, 5)]:
        m[node] = inp.unit_vector(rng)
    me = oracle_mod.Mesh(p.n, p.dx)
    me.set_material(*_material(p))
    ref = me.h_eff(m, oracle_mod.DEMAG)
    nodes = list(np.ndindex(*p.nodes))
    h = sampled.demag_at_nodes(p.n, p.dx, p.Ms_cells(), m, nodes)
    assert np.abs(ref).max() > 0
    np.testing.assert_allclose(h, ref.reshape(-1, 3), rtol=0, atol=1e-12 * np.abs(ref).max())
