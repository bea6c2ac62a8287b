"""Pins of the oracle's continuous adjoint (section "Inverse Micromagnetics", Eq. adjoint_system).

The dense LLG Jacobian is checked against central differences of the oracle's right-hand side, the
field Jacobian against the symmetry of the quadratic energies, and the adjoint gradients against
central differences of the forward loss: the continuous adjoint and the differentiated discrete forward
map both approach the exact gradient, so their gap shrinks with the fourth power of the step.
"""
import numpy as np
import pytest

import nm_inputs as inp
from helpers import oracle_mesh


@pytest.fixture(scope="module")
def oracle_adj():
    import oracle
    from oracle import adjoint
    return oracle, adjoint


def _problem(seed, shape=(2, 2, 1)):
    rng = np.random.default_rng(seed)
    p = inp.random_problem(rng, shape, vacuum=False)
    return p, rng


def _tangent(rng, m):
    d = rng.standard_normal(m.shape)
    d -= np.sum(d * m, axis=-1, keepdims=True) * m
    return d / np.linalg.norm(d)


def test_llg_jacobian_matches_central_differences(oracle_adj):
    oracle, adjoint = oracle_adj
    p, rng = _problem(1)
    me = oracle_mesh(oracle, p)
    ca = adjoint.ContinuousAdjoint(me, oracle.ALL)
    m = p.m0.reshape(-1)
    t = 3e-11
    J = ca.jacobian(m, t)
    for _ in range(4):
        d = rng.standard_normal(m.shape)
        eps = 1e-6
        fd = (ca.rhs(m + eps * d, t) - ca.rhs(m - eps * d, t)) / (2 * eps)
        assert np.linalg.norm(J @ d - fd) <= 1e-6 * np.linalg.norm(fd)


def test_field_jacobian_is_mass_symmetric(oracle_adj):
    """h_lin = -M^{-1} K with K symmetric: diag(mass) J_h is symmetric (Eqs. weak_form_discrete, mass_lumping)."""
    oracle, adjoint = oracle_adj
    p, _ = _problem(2, (3, 2, 2))
    me = oracle_mesh(oracle, p)
    ca = adjoint.ContinuousAdjoint(me, oracle.ALL)
    MJ = np.repeat(me.mass().reshape(-1), 3)[:, None] * ca.Jh
    assert np.abs(MJ - MJ.T).max() <= 1e-12 * np.abs(MJ).max()


def _loss(oracle, me, m0, T, n, W, tgt, renorm):
    m = m0.copy()
    h = T / n
    for k in range(n):
        m = me.rk4_step(m, k * h, h, oracle.ALL, renorm)
    return np.sum(W * (m - tgt) ** 2)


@pytest.mark.parametrize("renorm", [False, True])
def test_continuous_adjoint_converges_to_finite_differences(oracle_adj, renorm):
    oracle, adjoint = oracle_adj
    p, rng = _problem(3)
    me = oracle_mesh(oracle, p)
    ca = adjoint.ContinuousAdjoint(me, oracle.ALL)
    T = 2e-12
    W = rng.uniform(0.5, 1.5, p.m0.shape)
    tgt = inp.unit_vectors(rng, p.nodes)
    d = _tangent(rng, p.m0)
    errs = []
    for n in (8, 16, 32):
        loss, gm, gh, _ = ca.run(p.m0, 0.0, T, n, W, tgt, renorm, p.h_freq, p.h_phase)
        assert abs(loss - _loss(oracle, me, p.m0, T, n, W, tgt, renorm)) <= 1e-12 * loss
        eps = 1e-6
        fd = (_loss(oracle, me, p.m0 + eps * d, T, n, W, tgt, renorm)
              - _loss(oracle, me, p.m0 - eps * d, T, n, W, tgt, renorm)) / (2 * eps)
        errs.append(abs(np.sum(gm * d) - fd) / abs(fd))
    assert errs[-1] < 1e-4
    # fourth order: halving the step divides the gap by about 16
    assert errs[0] / errs[1] > 8 and errs[1] / errs[2] > 8


def test_field_gradient_converges_to_finite_differences(oracle_adj):
    """u(t0) for the uniform applied field against central differences in h (Eq. adjoint_system)."""
    oracle, adjoint = oracle_adj
    p, rng = _problem(4)
    T = 2e-12
    W = rng.uniform(0.5, 1.5, p.m0.shape)
    tgt = inp.unit_vectors(rng, p.nodes)
    errs = []
    for n in (8, 16, 32):
        me = oracle_mesh(oracle, p)
        ca = adjoint.ContinuousAdjoint(me, oracle.ALL)
        _, _, gh, _ = ca.run(p.m0, 0.0, T, n, W, tgt, True, p.h_freq, p.h_phase)
        dh = rng.standard_normal(3)
        dh *= 1e-3 * np.linalg.norm(p.h_uniform) / np.linalg.norm(dh)
        Ls = []
        for sgn in (1, -1):
            me2 = oracle_mesh(oracle, p)
            me2.set_zeeman(np.asarray(p.h_uniform) + sgn * dh, p.h_freq, p.h_phase, p.h_cell, p.cell_freq,
                           p.cell_phase)
            Ls.append(_loss(oracle, me2, p.m0, T, n, W, tgt, True))
        fd = (Ls[0] - Ls[1]) / 2
        errs.append(abs(gh @ dh - fd) / abs(fd))
    assert errs[-1] < 1e-4
    assert errs[0] / errs[1] > 8 and errs[1] / errs[2] > 8
