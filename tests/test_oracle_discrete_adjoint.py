"""Pins of the oracle's reference gradients of the discrete forward map (section "Automatic
Differentiation and Time Integration": backpropagation through the integrator with frozen steps;
Eq. inverse_min for the design variables).

The reverse-mode gradient (dense Jacobians, ``oracle.discrete_adjoint.DiscreteAdjoint``) and the
brute-force gradient (fourth-order central differences of the oracle's C steppers) are two routes that
share only the right-hand side; they must agree component by component.  The demag operator the
reverse route uses is checked against the oracle's direct demag sum, and a run without steps has the
closed-form gradient 2 W (m0 - target)."""
import numpy as np
import pytest

import nm_inputs as inp
from helpers import oracle_mesh


@pytest.fixture(scope="module")
def da():
    import oracle
    from oracle import discrete_adjoint
    return oracle, discrete_adjoint


def _setup(seed, shape=(3, 2, 2)):
    rng = np.random.default_rng(seed)
    p = inp.random_problem(rng, shape, vacuum=False)
    p.alpha = 0.2
    W = np.zeros(p.nodes + (3,))
    W[-2:, :, :, 1] = rng.uniform(0.5, 1.5, (2,) + p.nodes[1:])
    W[:, 0, :, 0] = 0.7
    tgt = inp.unit_vectors(rng, p.nodes) * 0.3
    return p, W, tgt, rng


def _factory(oracle, p):
    cache = {}

    def make_mesh(Ms):
        if "m" not in cache:
            cache["m"] = oracle_mesh(oracle, p)
        cache["m"].set_material(Ms, p.A_cells(), p.Ku_cells(), p.axis, p.alpha, p.gamma)
        return cache["m"]
    return make_mesh


def _zeeman(p):
    return (p.h_uniform, p.h_freq, p.h_phase, p.h_cell, p.cell_freq, p.cell_phase)


@pytest.mark.parametrize("method,renorm,initial", [(0, True, True), (1, True, False), (0, False, False),
                                                    (1, False, True)])
def test_reverse_gradient_matches_central_differences(da, method, renorm, initial):
    """Every component of dL/dMs and dL/dm0: reverse mode against four-point central differences of
    the oracle's own forward steps (all terms, heterogeneous material, time-harmonic uniform field and
    a cell field)."""
    oracle, d = da
    p, W, tgt, _ = _setup(5 + method + 2 * renorm)
    me = oracle_mesh(oracle, p)
    if method == d.RK4:
        plan = d.step_plan(me, p.m0, 0.0, 6e-14, d.RK4, 1e-14, sample_dt=2e-14, renorm=renorm)
    else:
        plan = d.step_plan(me, p.m0, 0.0, 6e-14, d.DP54, 5e-15, 1e-5, 1e-5, sample_dt=2e-14, renorm=renorm)
    assert len(plan) >= 3 and plan[-1][2]
    adj = d.DiscreteAdjoint(me, p.Ms_cells(), _zeeman(p), oracle.ALL)
    L, gMs, gm0 = adj.reverse_gradient(p.m0, plan, W, tgt, initial, method, renorm)
    assert L == pytest.approx(d.frozen_loss(me, p.m0, plan, W, tgt, initial, method, oracle.ALL, renorm),
                              rel=1e-13)
    fMs, fm0 = d.fd_gradient(_factory(oracle, p), p.Ms_cells(), p.m0, plan, W, tgt, initial, method,
                             oracle.ALL, renorm)
    assert np.abs(gMs - fMs).max() <= 1e-8 * np.abs(fMs).max()
    assert np.abs(gm0 - fm0).max() <= 1e-8 * np.abs(fm0).max()
    assert np.abs(fMs).max() > 0 and np.abs(fm0).max() > 0


def test_reverse_gradient_single_terms(da):
    """Each field term alone (the Ms derivative takes a different route for each).  Some terms give
    Ms gradients so small against the loss that the differences carry rounding of about
    1e-16 L / (1e-3 Ms) per component; the bar adds that floor."""
    oracle, d = da
    p, W, tgt, _ = _setup(11, (2, 2, 2))
    for terms in (oracle.EXCH, oracle.ANIS, oracle.ZEE, oracle.DEMAG):
        me = oracle_mesh(oracle, p)
        plan = d.step_plan(me, p.m0, 0.0, 4e-14, d.RK4, 1e-14, sample_dt=2e-14, terms=terms)
        adj = d.DiscreteAdjoint(me, p.Ms_cells(), _zeeman(p), terms)
        L, gMs, gm0 = adj.reverse_gradient(p.m0, plan, W, tgt, False, d.RK4)
        fMs, fm0 = d.fd_gradient(_factory(oracle, p), p.Ms_cells(), p.m0, plan, W, tgt, False, d.RK4, terms)
        assert np.abs(gm0 - fm0).max() <= 1e-8 * np.abs(fm0).max(), terms
        floor = 1e-12 * L / p.Ms_cells().min()
        assert np.abs(gMs - fMs).max() <= 1e-8 * np.abs(fMs).max() + floor, terms


def test_no_steps_closed_form(da):
    """A run without steps, loss at t0 only: dL/dm0 = 2 W (m0 - target), dL/dMs = 0."""
    oracle, d = da
    p, W, tgt, _ = _setup(12)
    me = oracle_mesh(oracle, p)
    adj = d.DiscreteAdjoint(me, p.Ms_cells(), _zeeman(p), oracle.ALL)
    L, gMs, gm0 = adj.reverse_gradient(p.m0, [], W, tgt, True, d.DP54)
    assert L == pytest.approx(np.sum(W * (p.m0 - tgt) ** 2), rel=1e-15)
    assert np.array_equal(gm0, 2.0 * W * (p.m0 - tgt))
    assert not np.any(gMs)


def test_demag_operator_reproduces_direct_sum(da):
    """G (Ms mbar) equals the oracle's direct demag sum for a random state; G is symmetric (the
    Newell tensor is even in the offset and symmetric)."""
    oracle, d = da
    p, _, _, rng = _setup(13, (3, 2, 2))
    me = oracle_mesh(oracle, p)
    G = d.demag_operator(p.n, p.dx)
    nc = int(np.prod(p.n))
    M = (p.Ms_cells()[..., None] * d.cell_mean(p.m0)).reshape(nc * 3)
    H = (G.reshape(nc * 3, nc * 3) @ M).reshape(p.n + (3,))
    ref = me.demag_cells(p.m0)
    assert np.abs(H - ref).max() <= 1e-13 * np.abs(ref).max()
    G2 = G.reshape(nc * 3, nc * 3)
    assert np.abs(G2 - G2.T).max() <= 1e-14 * np.abs(G2).max()


def test_step_plan_lands_on_sample_times(da):
    """Accepted steps chain without gaps, sample ends fall on t0 + k sample_dt, and the Dormand-Prince
    plan reproduces the adaptive run's state when replayed with the steps frozen."""
    oracle, d = da
    p, W, tgt, _ = _setup(14)
    me = oracle_mesh(oracle, p)
    plan = d.step_plan(me, p.m0, 0.0, 1e-13, d.DP54, 3e-15, 1e-6, 1e-6, sample_dt=2.5e-14)
    t = 0.0
    k = 1
    for ts, dt, is_sample in plan:
        assert ts == t
        t = ts + dt
        if is_sample:
            assert abs(t - k * 2.5e-14) <= 1e-12 * 1e-13 + 1e-9 * 2.5e-14
            k += 1
    assert k == 5
    st = me.dp5_stepper(p.m0, 0.0, 3e-15, oracle.ALL, 1e-6, 1e-6)
    # the adaptive run accepts each planned step at its planned size
    for ts, dt, _ in plan:
        st.t.value = ts
        st.set_dt(dt)
        assert st.step()
    Wl = np.zeros_like(W)
    Wl[..., :] = 1.0
    last = d.frozen_loss(me, p.m0, [(a, b, i == len(plan) - 1) for i, (a, b, _) in enumerate(plan)], Wl, None)
    assert last == pytest.approx(np.sum(st.m ** 2), rel=1e-14)
