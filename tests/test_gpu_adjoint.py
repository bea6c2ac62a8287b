"""Gradients on the GPU: the effective-field transpose product against the oracle (exact for the
m-gradient, central differences for the Ms-gradient), and the discrete adjoint of RK4 / Dormand-Prince
integration against central finite differences of the loss with the step sizes frozen."""
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


def _vjp(nmgb, p, precision, m, v, t):
    import torch
    me = gpu_mesh(nmgb, p, precision)
    gm, gMs = me.h_eff_vjp(torch.tensor(m, dtype=me.dtype, device="cuda"),
                           torch.tensor(v, dtype=me.dtype, device="cuda"), p.terms, t)
    out = gm.double().cpu().numpy(), gMs.double().cpu().numpy()
    me.close()
    return out


@pytest.mark.parametrize("precision,tol", [(1, 1e-10), (0, 1e-4)])
def test_heff_vjp_m_matches_oracle(oracle_mod, nmgb, precision, tol):
    """<v, h(m)> is affine in m, so each component of the gradient is an exact difference."""
    rng = np.random.default_rng(31)
    p = inp.random_problem(rng, (4, 3, 2), vacuum=True)
    m = p.m0.astype(np.float32).astype(np.float64)
    v = rng.standard_normal(p.nodes + (3,)).astype(np.float32).astype(np.float64)
    t = 0.4e-9
    ref = oracle_mesh(oracle_mod, p)
    L0 = np.sum(v * ref.h_eff(m, oracle_mod.ALL, t))
    g_ref = np.zeros_like(m)
    for idx in np.ndindex(*m.shape):
        e = m.copy()
        e[idx] += 1.0
        g_ref[idx] = np.sum(v * ref.h_eff(e, oracle_mod.ALL, t)) - L0
    gm, _ = _vjp(nmgb, p, precision, m, v, t)
    assert rel_l2(gm, g_ref) < tol


@pytest.mark.parametrize("precision,tol", [(1, 1e-7), (0, 2e-4)])
def test_heff_vjp_Ms_matches_oracle_differences(oracle_mod, nmgb, precision, tol):
    rng = np.random.default_rng(32)
    p = inp.random_problem(rng, (4, 3, 2), vacuum=False)
    p.h_freq = 2e9
    m = p.m0.astype(np.float32).astype(np.float64)
    v = rng.standard_normal(p.nodes + (3,)).astype(np.float32).astype(np.float64)
    t = 0.3e-9
    Ms = p.Ms_cells()
    g_ref = np.zeros(p.n)
    for c in np.ndindex(*p.n):
        vals = []
        for sgn in (1, -1):
            q = inp.Problem(**{**p.__dict__})
            M2 = Ms.copy()
            M2[c] += sgn * 1e-4 * Ms[c]
            q.Ms = M2
            vals.append(np.sum(v * oracle_mesh(oracle_mod, q).h_eff(m, oracle_mod.ALL, t)))
        g_ref[c] = (vals[0] - vals[1]) / (2e-4 * Ms[c])
    _, gMs = _vjp(nmgb, p, precision, m, v, t)
    assert rel_l2(gMs, g_ref) < tol


def _loss_problem(seed, n=(6, 5, 2)):
    rng = np.random.default_rng(seed)
    p = inp.random_problem(rng, n, heterogeneous=True, vacuum=False)
    p.h_freq = 0.0
    p.alpha = 0.2
    W = np.zeros(p.nodes + (3,))
    W[-3:, :, :, 1] = rng.uniform(0.5, 1.5, (3,) + p.nodes[1:])
    tgt = inp.unit_vectors(rng, p.nodes) * 0.3
    return p, W, tgt, rng


def _run(nmgb, p, Ms, W, tgt, kw):
    me = gpu_mesh(nmgb, p, 1)
    me.set_material(Ms, p.A_cells(), p.Ku_cells(), p.axis, p.alpha, p.gamma)
    me.set_state(kw.pop("m0", p.m0), 0.0, 1e-14)
    out = me.adjoint_run(weight=W, target=tgt, **kw)
    me.close()
    return out


@pytest.mark.parametrize("method", ["RK4", "DP54"])
def test_adjoint_matches_finite_differences(nmgb, method):
    """Frozen step sizes: RK4 with a fixed step; Dormand-Prince with tolerances so loose that every
    attempt is accepted and the steps are set by the clipping to the sample times alone."""
    p, W, tgt, rng = _loss_problem(40)
    Ms = p.Ms_cells()
    if method == "RK4":
        kw = dict(t_end=1.2e-13, method=nmgb.RK4, dt0=1e-14, sample_dt=3e-14, include_initial=True,
                  checkpoint_every=3)
    else:
        kw = dict(t_end=1.2e-13, method=nmgb.DP54, rtol=1e3, atol=1e3, dt0=5e-15, sample_dt=2e-14,
                  checkpoint_every=4)
    loss, gMs, gm0, nst = _run(nmgb, p, Ms, W, tgt, dict(kw))
    assert nst >= 4 and loss > 0
    for _ in range(3):
        d = rng.standard_normal(p.n) * Ms * 1e-5
        lp = _run(nmgb, p, Ms + d, W, tgt, dict(kw))[0]
        lm = _run(nmgb, p, Ms - d, W, tgt, dict(kw))[0]
        fd = (lp - lm) / 2
        ad = np.sum(gMs * d)
        assert abs(fd - ad) <= 1e-6 * abs(fd) + 1e-12 * loss, (fd, ad)
    d = rng.standard_normal(p.nodes + (3,)) * 1e-6
    lp = _run(nmgb, p, Ms, W, tgt, dict(kw, m0=p.m0 + d))[0]
    lm = _run(nmgb, p, Ms, W, tgt, dict(kw, m0=p.m0 - d))[0]
    fd = (lp - lm) / 2
    ad = np.sum(gm0 * d)
    assert abs(fd - ad) <= 1e-5 * abs(fd) + 1e-12 * loss, (fd, ad)


def test_adjoint_checkpoint_interval_does_not_change_gradient(nmgb):
    p, W, tgt, _ = _loss_problem(41)
    kw = dict(t_end=1e-13, method=nmgb.DP54, rtol=1e-4, atol=1e-4, dt0=1e-14, sample_dt=2.5e-14)
    a = _run(nmgb, p, p.Ms_cells(), W, tgt, dict(kw, checkpoint_every=1))
    b = _run(nmgb, p, p.Ms_cells(), W, tgt, dict(kw, checkpoint_every=1000))
    assert a[0] == b[0] and a[3] == b[3]
    assert rel_l2(a[1], b[1]) < 1e-13 and rel_l2(a[2], b[2]) < 1e-13


def test_field_gradient_matches_finite_differences(nmgb):
    """dL/dh of the uniform applied field (frozen step sizes) against central differences."""
    p, W, tgt, rng = _loss_problem(42)
    p.h_freq = 0.0
    kw = dict(t_end=1.2e-13, method=nmgb.DP54, rtol=1e3, atol=1e3, dt0=5e-15, sample_dt=2e-14, checkpoint_every=4)

    def run(h, field_grad=False):
        me = gpu_mesh(nmgb, p, 1)
        me.set_uniform_field(h)
        me.set_state(p.m0, 0.0, 1e-14)
        out = me.adjoint_run(weight=W, target=tgt, field_grad=field_grad, **kw)
        me.close()
        return out

    h0 = np.array(p.h_uniform)
    loss, _, _, _, gh = run(h0, True)
    assert loss > 0 and np.abs(gh).max() > 0
    for _ in range(3):
        d = rng.standard_normal(3) * 1e-3 * np.linalg.norm(h0)
        fd = (run(h0 + d)[0] - run(h0 - d)[0]) / 2
        assert abs(fd - gh @ d) <= 1e-6 * abs(fd) + 1e-12 * loss, (fd, gh @ d)
