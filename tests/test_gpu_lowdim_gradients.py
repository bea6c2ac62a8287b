"""Gradients on the 2D and 1D nodal bases (section "Low-Dimensional Geometries" with section "Inverse
Micromagnetics"): the effective-field transpose product against the oracle's restricted system (exact
differences for the m-gradient, central differences for the Ms-gradient), the discrete adjoint against
central finite differences of the loss with the step sizes frozen, and the continuous adjoint's
convergence to the discrete one."""
import numpy as np
import pytest

import nm_inputs as inp
from helpers import rel_l2

pytestmark = pytest.mark.gpu

SHAPE = {2: (4, 3, 2), 1: (5, 2, 3)}


@pytest.fixture(scope="module")
def nmgb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_11725_gb300 as nmgb
    nmgb.load()
    return nmgb


def _nodes(p, basis):
    return (p.n[0] + 1, 1 if basis == 1 else p.n[1] + 1, 1)


def _oracle(p, basis, Ms=None):
    from oracle import basis1d, basis2d
    me = (basis2d.Mesh2D if basis == 2 else basis1d.Mesh1D)(p.n, p.dx)
    me.set_material(p.Ms_cells() if Ms is None else Ms, p.A_cells(), p.Ku_cells(), p.axis, p.alpha, p.gamma)
    me.set_zeeman(p.h_uniform, p.h_freq, p.h_phase, p.h_cell, p.cell_freq, p.cell_phase)
    return me


def _gpu(nmgb, p, basis, precision, Ms=None):
    me = nmgb.Mesh(p.n, p.dx, precision, basis=basis)
    me.set_material(p.Ms_cells() if Ms is None else Ms, p.A_cells(), p.Ku_cells(), p.axis, p.alpha, p.gamma)
    me.set_zeeman(p.h_uniform, p.h_freq, p.h_phase, p.h_cell, p.cell_freq, p.cell_phase)
    me.set_terms(p.terms)
    return me


def _vjp(nmgb, p, basis, precision, m, v, t):
    import torch
    me = _gpu(nmgb, p, basis, precision)
    gm, gMs = me.h_eff_vjp(torch.tensor(m, dtype=me.dtype, device="cuda"),
                           torch.tensor(v, dtype=me.dtype, device="cuda"), p.terms, t)
    out = gm.double().cpu().numpy(), gMs.double().cpu().numpy()
    me.close()
    return out


@pytest.mark.parametrize("basis", [2, 1])
@pytest.mark.parametrize("precision,tol", [(1, 1e-10), (0, 1e-4)])
def test_heff_vjp_m_matches_oracle(oracle_mod, nmgb, basis, precision, tol):
    """<v, h(m)> is affine in m, so each component of the gradient is an exact difference."""
    rng = np.random.default_rng(51 + basis)
    p = inp.random_problem(rng, SHAPE[basis], vacuum=True)
    nodes = _nodes(p, basis)
    m = inp.unit_vectors(rng, nodes).astype(np.float32).astype(np.float64)
    v = rng.standard_normal(nodes + (3,)).astype(np.float32).astype(np.float64)
    t = 0.4e-9
    ref = _oracle(p, basis)
    L0 = np.sum(v * ref.h_eff(m, oracle_mod.ALL, t))
    g_ref = np.zeros_like(m)
    for idx in np.ndindex(*m.shape):
        e = m.copy()
        e[idx] += 1.0
        g_ref[idx] = np.sum(v * ref.h_eff(e, oracle_mod.ALL, t)) - L0
    gm, _ = _vjp(nmgb, p, basis, precision, m, v, t)
    assert gm.shape == m.shape
    assert rel_l2(gm, g_ref) < tol


@pytest.mark.parametrize("basis", [2, 1])
@pytest.mark.parametrize("precision,tol", [(1, 1e-7), (0, 2e-4)])
def test_heff_vjp_Ms_matches_oracle_differences(oracle_mod, nmgb, basis, precision, tol):
    rng = np.random.default_rng(53 + basis)
    p = inp.random_problem(rng, SHAPE[basis], vacuum=False)
    p.h_freq = 2e9
    nodes = _nodes(p, basis)
    m = inp.unit_vectors(rng, nodes).astype(np.float32).astype(np.float64)
    v = rng.standard_normal(nodes + (3,)).astype(np.float32).astype(np.float64)
    t = 0.3e-9
    Ms = p.Ms_cells()
    g_ref = np.zeros(p.n)
    for c in np.ndindex(*p.n):
        vals = []
        for sgn in (1, -1):
            M2 = Ms.copy()
            M2[c] += sgn * 1e-4 * Ms[c]
            vals.append(np.sum(v * _oracle(p, basis, M2).h_eff(m, oracle_mod.ALL, t)))
        g_ref[c] = (vals[0] - vals[1]) / (2e-4 * Ms[c])
    _, gMs = _vjp(nmgb, p, basis, precision, m, v, t)
    assert rel_l2(gMs, g_ref) < tol


def _loss_problem(seed, basis):
    rng = np.random.default_rng(seed)
    p = inp.random_problem(rng, SHAPE[basis], heterogeneous=True, vacuum=False)
    p.h_freq = 0.0
    p.alpha = 0.2
    nodes = _nodes(p, basis)
    W = rng.uniform(0.5, 1.5, nodes + (3,))
    tgt = inp.unit_vectors(rng, nodes) * 0.3
    m0 = inp.unit_vectors(rng, nodes)
    return p, W, tgt, m0, rng


@pytest.mark.parametrize("basis", [2, 1])
def test_discrete_adjoint_matches_finite_differences(nmgb, basis):
    """RK4 with a fixed step (frozen step sizes): Ms-map and m0 directions."""
    p, W, tgt, m0, rng = _loss_problem(60 + basis, basis)
    Ms = p.Ms_cells()
    kw = dict(t_end=1.2e-13, method=nmgb.RK4, dt0=1e-14, sample_dt=3e-14, include_initial=True,
              checkpoint_every=3)

    def run(Ms_, m0_):
        me = _gpu(nmgb, p, basis, 1, Ms_)
        me.set_state(m0_, 0.0, 1e-14)
        out = me.adjoint_run(weight=W, target=tgt, **kw)
        me.close()
        return out

    loss, gMs, gm0, nst = run(Ms, m0)
    assert nst >= 4 and loss > 0 and gm0.shape == m0.shape
    for _ in range(2):
        d = rng.standard_normal(p.n) * Ms * 1e-5
        fd = (run(Ms + d, m0)[0] - run(Ms - d, m0)[0]) / 2
        ad = np.sum(gMs * d)
        assert abs(fd - ad) <= 1e-6 * abs(fd) + 1e-12 * loss, (fd, ad)
    d = rng.standard_normal(m0.shape) * 1e-6
    fd = (run(Ms, m0 + d)[0] - run(Ms, m0 - d)[0]) / 2
    ad = np.sum(gm0 * d)
    assert abs(fd - ad) <= 1e-5 * abs(fd) + 1e-12 * loss, (fd, ad)


@pytest.mark.parametrize("basis,steps", [(2, (8, 16, 32)), (1, (16, 32, 64))])
def test_continuous_adjoint_converges_to_discrete(nmgb, basis, steps):
    """The m0, Ms-map and uniform-field gradients of the continuous adjoint approach the discrete
    adjoint's with the fourth power of the step.  Each problem is taken over step counts in its
    asymptotic range (the 1D-basis problem's error constant is larger: 0.38 at 8 steps)."""
    p, W, tgt, m0, _ = _loss_problem(70 + basis, basis)
    T = 2e-12
    errs = {"m0": [], "Ms": [], "h": []}
    for n in steps:
        me = _gpu(nmgb, p, basis, 1)
        me.set_state(m0, 0.0, 1e-14)
        _, gm, gMs, gh, _ = me.adjoint_continuous(T, n, W, tgt)
        me.close()
        me = _gpu(nmgb, p, basis, 1)
        me.set_state(m0, 0.0, 1e-14)
        _, dMs, dm0, ns, dh = me.adjoint_run(T, W, tgt, method=nmgb.RK4, dt0=T / n, field_grad=True)
        me.close()
        assert ns == n

        def tang(g):
            return g - np.sum(g * m0, -1, keepdims=True) * m0
        errs["m0"].append(rel_l2(tang(gm), tang(dm0)))
        errs["Ms"].append(rel_l2(gMs, dMs))
        errs["h"].append(rel_l2(gh, dh))
    for k, e in errs.items():
        assert e[-1] < 1e-4, (k, e)
        assert e[0] / e[1] > 8 and e[1] / e[2] > 8, (k, e)
