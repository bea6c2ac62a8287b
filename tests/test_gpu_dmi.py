"""Interfacial DMI on the GPU (nm_set_dmi, term bit NM_DMI) against the oracle: the field alone and with
every other term, the transpose product, and RK4 trajectories.  FP64 rel-L2 <= 1e-12, FP32 <= 1e-5.
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


def _setup(oracle_mod, nmgb, shape, precision, seed, vacuum, D_map):
    rng = np.random.default_rng(seed)
    p = inp.random_problem(rng, shape, vacuum=vacuum)
    D = rng.uniform(-3e-3, 3e-3, p.n) if D_map else 2.5e-3
    om = oracle_mesh(oracle_mod, p)
    om.set_dmi(D)
    gm = gpu_mesh(nmgb, p, precision)
    gm.set_dmi(D)
    return p, om, gm, rng


def _h(me, m, terms, t):
    import torch
    return me.h_eff(torch.tensor(m, dtype=me.dtype, device="cuda"), terms, t).double().cpu().numpy()


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("shape,vacuum,D_map", [((5, 4, 3), False, False), ((13, 7, 5), True, True),
                                                ((16, 16, 4), False, True), ((9, 1, 2), True, False)])
def test_field_matches_oracle(oracle_mod, nmgb, precision, shape, vacuum, D_map):
    p, om, gm, rng = _setup(oracle_mod, nmgb, shape, precision, 21, vacuum, D_map)
    m = rounded(p.m0, precision)
    for terms in (oracle_mod.DMI, oracle_mod.ALL | oracle_mod.DMI):
        ref = om.h_eff(m, terms, 0.9e-10)
        h = _h(gm, m, terms, 0.9e-10)
        assert rel_l2(h, ref) < TOL[precision], terms
    # without the bit the term is off
    assert rel_l2(_h(gm, m, oracle_mod.ALL, 0.9e-10), om.h_eff(m, oracle_mod.ALL, 0.9e-10)) < TOL[precision]
    gm.close()


def test_transpose_product_includes_dmi(oracle_mod, nmgb):
    """J_h^T v = -K (v / mass) with the DMI part of K (a symmetric quadratic form)."""
    import torch
    p, om, gm, rng = _setup(oracle_mod, nmgb, (4, 3, 2), 1, 22, True, True)
    terms = oracle_mod.DMI | oracle_mod.EXCH
    v = rng.standard_normal(p.nodes + (3,))
    mass = om.mass()[..., None]
    w = np.where(mass > 0, v / np.where(mass > 0, mass, 1.0), 0.0)
    ref = -om.variation(w, terms, 0.0)
    mt = torch.tensor(p.m0, device="cuda")
    g, _ = gm.h_eff_vjp(mt, torch.tensor(v, device="cuda"), terms, 0.0, want_Ms=False)
    assert rel_l2(g.cpu().numpy(), ref) < 1e-12
    gm.close()


def test_rk4_trajectory_with_dmi(oracle_mod, nmgb):
    p, om, gm, rng = _setup(oracle_mod, nmgb, (8, 6, 3), 1, 23, False, True)
    terms = oracle_mod.ALL | oracle_mod.DMI
    gm.set_terms(terms)
    steps, dt = 25, 1e-14
    ref = p.m0.copy()
    for s in range(steps):
        ref = om.rk4_step(ref, s * dt, dt, terms, renorm=True)
    gm.set_state(p.m0, 0.0, dt)
    gm.run_steps(steps, nmgb.RK4, 0.0, 0.0)
    m, _, _ = gm.get_state()
    assert rel_l2(m, ref) < 1e-12
    gm.close()


def test_dmi_needs_the_3d_basis(nmgb):
    me = nmgb.Mesh((4, 4, 1), (2e-9, 2e-9, 2e-9), nmgb.F64, basis=2)
    with pytest.raises(nmgb.NMError):
        me.set_dmi(1e-3)
    me.close()
