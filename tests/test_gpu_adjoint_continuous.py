"""Continuous adjoint-state gradients on the GPU (nm_adjoint_continuous, section "Inverse
Micromagnetics", Eq. adjoint_system): parity with the oracle's backward integration, and convergence
to the discrete adjoint (the exact gradient of the forward map) with the fourth power of the step.
"""
import numpy as np
import pytest

import nm_inputs as inp
from helpers import gpu_mesh, oracle_mesh, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nmgb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_11725_gb300 as nmgb
    nmgb.load()
    return nmgb


def _problem(seed, shape):
    rng = np.random.default_rng(seed)
    p = inp.random_problem(rng, shape, vacuum=False)
    W = rng.uniform(0.5, 1.5, p.m0.shape)
    tgt = inp.unit_vectors(rng, p.nodes)
    return p, W, tgt, rng


@pytest.mark.parametrize("precision,tol", [(1, 1e-9), (0, 2e-3)])
@pytest.mark.parametrize("shape", [(2, 2, 1), (3, 2, 2)])
def test_matches_oracle(oracle_mod, nmgb, precision, tol, shape):
    from oracle import adjoint
    p, W, tgt, _ = _problem(11, shape)
    T, n = 2e-12, 16
    ca = adjoint.ContinuousAdjoint(oracle_mesh(oracle_mod, p), oracle_mod.ALL)
    loss_r, gm_r, gh_r, m0_r = ca.run(p.m0, 0.0, T, n, W, tgt, True, p.h_freq, p.h_phase)
    me = gpu_mesh(nmgb, p, precision)
    me.set_state(p.m0, 0.0, 1e-14)
    loss, gm, gMs, gh, m0r = me.adjoint_continuous(T, n, W, tgt)
    assert abs(loss - loss_r) <= tol * loss_r
    assert rel_l2(gm, gm_r) < tol
    assert rel_l2(gh, gh_r) < tol
    assert rel_l2(m0r, m0_r) < tol
    m, t, _ = me.get_state()
    assert abs(t - T) <= 1e-9 * T
    me.close()


def test_converges_to_discrete_adjoint(nmgb):
    """All three gradients (m0, Ms map, uniform field) approach the discrete adjoint's as the step halves."""
    p, W, tgt, _ = _problem(12, (3, 2, 2))
    T = 2e-12
    errs = {"m0": [], "Ms": [], "h": []}
    for n in (8, 16, 32):
        me = gpu_mesh(nmgb, p, 1)
        me.set_state(p.m0, 0.0, 1e-14)
        _, gm, gMs, gh, _ = me.adjoint_continuous(T, n, W, tgt)
        me.close()
        me = gpu_mesh(nmgb, p, 1)
        me.set_state(p.m0, 0.0, 1e-14)
        _, dMs, dm0, ns, dh = me.adjoint_run(T, W, tgt, method=nmgb.RK4, dt0=T / n, field_grad=True)
        me.close()
        assert ns == n
        # the tangential part of the m0 gradient (renormalisation removes the radial one in the discrete map)
        def tang(g):
            return g - np.sum(g * p.m0, -1, keepdims=True) * p.m0
        errs["m0"].append(rel_l2(tang(gm), tang(dm0)))
        errs["Ms"].append(rel_l2(gMs, dMs))
        errs["h"].append(rel_l2(gh, dh))
    for k, e in errs.items():
        assert e[-1] < 1e-4, (k, e)
        assert e[0] / e[1] > 8 and e[1] / e[2] > 8, (k, e)


def test_reconstruction_error_shrinks(nmgb):
    """The backward integration reconstructs m(t0); its error falls with the step (section "Inverse
    Micromagnetics": the reduced accuracy of the reconstructed trajectory)."""
    p, W, tgt, _ = _problem(13, (2, 2, 1))
    T = 2e-12
    e = []
    for n in (8, 16):
        me = gpu_mesh(nmgb, p, 1)
        me.set_state(p.m0, 0.0, 1e-14)
        *_, m0r = me.adjoint_continuous(T, n, W, tgt)
        me.close()
        e.append(np.abs(m0r - p.m0).max())
    assert e[1] < e[0] / 8 and e[1] < 1e-3


def test_arguments(nmgb):
    p, W, tgt, _ = _problem(14, (2, 1, 1))
    me = gpu_mesh(nmgb, p, 1)
    with pytest.raises(nmgb.NMError):
        me.adjoint_continuous(1e-12, 4, W, tgt)  # no resident state
    me.set_state(p.m0, 0.0, 1e-14)
    with pytest.raises(nmgb.NMError):
        me.adjoint_continuous(1e-12, 0, W, tgt)
    with pytest.raises(nmgb.NMError):
        me.adjoint_continuous(-1e-12, 4, W, tgt)
    me.close()
