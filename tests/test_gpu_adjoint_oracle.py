"""The GPU's discrete adjoint (nm_adjoint_run) against the oracle's gradient of the same discrete forward
map (section "Automatic Differentiation and Time Integration"; Eq. inverse_min for the design
variables): dL/dMs of the cell Ms map and dL/dm0, component by component, for RK4 and Dormand-Prince
on 6x5x2 and 16x8x1 cells.

The reference never comes from the GPU: the oracle plans the steps itself (the same clipping to the
sample times and the same controller), and its gradient is the reverse sweep through dense Jacobians,
which the CPU tests pin to central differences of the oracle's forward runs.  A few components are also
compared with those central differences directly.

Bars:
  * FP64: relative L2 <= 1e-9 on each gradient, max component error <= 1e-8 of the largest component.
    The two sides differ only by rounding in FP64 (step sizes agree to ~1e-16 relative).
  * FP32 (FP32 field evaluations and slopes, FP64 state and accumulators): relative L2 <= 2e-4.  The
    FP32 field carries relative errors of ~1e-6 per evaluation, which the adjoint's transpose products
    and the forward recomputation repeat over every stage.
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


@pytest.fixture(scope="module")
def da():
    import oracle
    from oracle import discrete_adjoint
    return oracle, discrete_adjoint


def _problem(seed, shape):
    rng = np.random.default_rng(seed)
    p = inp.random_problem(rng, shape, heterogeneous=True, vacuum=False)
    p.alpha = 0.2
    W = np.zeros(p.nodes + (3,))
    W[-3:, :, :, 1] = rng.uniform(0.5, 1.5, (3,) + p.nodes[1:])
    W[:, 0, :, 0] = 0.5
    tgt = inp.unit_vectors(rng, p.nodes) * 0.3
    return p, W, tgt, rng


def _gpu(nmgb, p, precision, W, tgt, kw):
    me = gpu_mesh(nmgb, p, precision)
    me.set_state(p.m0, 0.0, kw["dt0"])
    out = me.adjoint_run(weight=W, target=tgt, **kw)
    me.close()
    return out


# (method, precision, keyword arguments of the run).  The FP64 Dormand-Prince case adapts its steps and
# rejects one attempt (8 and 10 accepted steps on the two meshes); FP32 Dormand-Prince takes tolerances
# so loose that every attempt is accepted, which fixes the step sizes independently of FP32 error norms.
CASES = [
    ("RK4", 1, dict(t_end=1.5e-13, dt0=1e-14, sample_dt=3e-14, include_initial=True, checkpoint_every=4)),
    ("DP54", 1, dict(t_end=3e-13, dt0=1.5e-13, sample_dt=1.5e-13, rtol=1e-9, atol=1e-9, checkpoint_every=3)),
    ("RK4", 0, dict(t_end=1.5e-13, dt0=1e-14, sample_dt=3e-14, include_initial=True, checkpoint_every=4)),
    ("DP54", 0, dict(t_end=1.5e-13, dt0=5e-15, sample_dt=3e-14, rtol=1e3, atol=1e3, checkpoint_every=3)),
]


@pytest.mark.parametrize("shape", [(6, 5, 2), (16, 8, 1)])
@pytest.mark.parametrize("method,precision,kw", CASES)
def test_discrete_adjoint_matches_oracle_gradient(nmgb, da, shape, method, precision, kw):
    oracle, d = da
    p, W, tgt, _ = _problem(40 + shape[0], shape)
    om = d.RK4 if method == "RK4" else d.DP54
    gkw = dict(kw, method=getattr(nmgb, method))
    loss, gMs, gm0, nst = _gpu(nmgb, p, precision, W, tgt, dict(gkw))
    me = oracle_mesh(oracle, p)
    plan = d.step_plan(me, p.m0, 0.0, kw["t_end"], om, kw["dt0"], kw.get("rtol", 1e-5), kw.get("atol", 1e-5),
                       kw["sample_dt"])
    assert nst == len(plan) >= 4
    adj = d.DiscreteAdjoint(me, p.Ms_cells(), (p.h_uniform, p.h_freq, p.h_phase, p.h_cell, p.cell_freq,
                                                p.cell_phase), oracle.ALL)
    L, rMs, rm0 = adj.reverse_gradient(p.m0, plan, W, tgt, kw.get("include_initial", False), om)
    if precision == 1:
        assert loss == pytest.approx(L, rel=1e-12)
        for g, r in ((gMs, rMs), (gm0, rm0)):
            assert rel_l2(g, r) <= 1e-9
            assert np.abs(g - r).max() <= 1e-8 * np.abs(r).max()
    else:
        assert loss == pytest.approx(L, rel=1e-5)
        assert rel_l2(gMs, rMs) <= 2e-4
        assert rel_l2(gm0, rm0) <= 2e-4


@pytest.mark.parametrize("method", ["RK4", "DP54"])
def test_discrete_adjoint_matches_oracle_central_differences(nmgb, da, method):
    """Sampled components against brute-force central differences of the oracle's own forward runs."""
    oracle, d = da
    p, W, tgt, rng = _problem(61, (6, 5, 2))
    kw = CASES[0][2] if method == "RK4" else CASES[1][2]
    om = d.RK4 if method == "RK4" else d.DP54
    _, gMs, gm0, _ = _gpu(nmgb, p, 1, W, tgt, dict(kw, method=getattr(nmgb, method)))
    me = oracle_mesh(oracle, p)
    plan = d.step_plan(me, p.m0, 0.0, kw["t_end"], om, kw["dt0"], kw.get("rtol", 1e-5), kw.get("atol", 1e-5),
                       kw["sample_dt"])
    cells = [tuple(int(rng.integers(0, s)) for s in p.n) for _ in range(8)]
    comps = [tuple(int(rng.integers(0, s)) for s in p.nodes + (3,)) for _ in range(8)]

    cache = {}

    def make_mesh(Ms):
        if "m" not in cache:
            cache["m"] = oracle_mesh(oracle, p)
        cache["m"].set_material(Ms, p.A_cells(), p.Ku_cells(), p.axis, p.alpha, p.gamma)
        return cache["m"]
    fMs, fm0 = d.fd_gradient(make_mesh, p.Ms_cells(), p.m0, plan, W, tgt, kw.get("include_initial", False), om,
                             oracle.ALL, True, ms_cells=cells, m0_components=comps)
    sMs = np.abs(gMs).max()
    sm0 = np.abs(gm0).max()
    for c in cells:
        assert abs(gMs[c] - fMs[c]) <= 1e-7 * sMs, (c, gMs[c], fMs[c])
    for c in comps:
        assert abs(gm0[c] - fm0[c]) <= 1e-7 * sm0, (c, gm0[c], fm0[c])
