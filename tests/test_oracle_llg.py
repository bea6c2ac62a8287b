"""Pins of the oracle's LLG right-hand side (Eq. llg) and its integrators (RK4, Dormand-Prince 5(4)).

References: the closed-form macrospin precession under a static field, the Runge-Kutta order
conditions of the published Dormand-Prince coefficients, the observed convergence order, and the
invariants of the LLG equation (|m| = 1, energy conservation at alpha = 0, dissipation for alpha > 0).
"""
from fractions import Fraction

import numpy as np
import pytest

import nm_inputs as inp

MU0 = 4e-7 * np.pi


def macrospin(oracle_mod, alpha, H, Ms=8e5):
    """A single cubic cell: its demag field is -Ms m/3, parallel to m, so only the applied field acts.
    A = 0: with identical nodes exchange vanishes anyway, and leaving it out keeps the stiff exchange
    modes from amplifying rounding differences between the nodes at large steps."""
    me = oracle_mod.Mesh((1, 1, 1), (3e-9, 3e-9, 3e-9))
    me.set_material(Ms, 0.0, 0.0, (0, 0, 1), alpha, inp.GAMMA)
    me.set_zeeman((0.0, 0.0, H))
    return me


def exact_macrospin(theta0, phi0, alpha, H, t):
    g = inp.GAMMA / (1 + alpha ** 2)
    th = 2 * np.arctan(np.tan(theta0 / 2) * np.exp(-alpha * g * H * t))
    ph = phi0 + g * H * t
    return np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])




def test_macrospin_closed_form_rk4(oracle_mod):
    alpha, H = 0.1, 8e4
    me = macrospin(oracle_mod, alpha, H)
    th0, ph0 = 2.5, 0.3
    m0 = np.array([np.sin(th0) * np.cos(ph0), np.sin(th0) * np.sin(ph0), np.cos(th0)])
    m = np.broadcast_to(m0, (2, 2, 2, 3)).copy()
    dt, steps = 2e-13, 100
    for s in range(steps):
        m = me.rk4_step(m, s * dt, dt, oracle_mod.ALL)
    ref = exact_macrospin(th0, ph0, alpha, H, steps * dt)
    assert np.abs(m - ref).max() < 1e-9


def test_llg_rhs_orthogonal_and_sign(oracle_mod):
    rng = np.random.default_rng(20)
    p = inp.random_problem(rng, (3, 2, 2))
    me = oracle_mod.Mesh(p.n, p.dx)
    me.set_material(p.Ms_cells(), p.A_cells(), p.Ku_cells(), p.axis, 0.0, p.gamma)
    me.set_zeeman(p.h_uniform)
    m = p.m0
    k = me.llg_rhs(m)
    H = me.h_eff(m)
    # dm/dt is orthogonal to m, and for alpha = 0 also to H: -gamma m x H
    assert np.abs(np.sum(k * m, -1)).max() < 1e-12 * np.abs(k).max()
    assert np.abs(k + inp.GAMMA * np.cross(m, H)).max() < 1e-12 * np.abs(k).max()


def _rk_order_conditions(c, a, b, order):
    A = [[Fraction(x).limit_denominator(10 ** 9) for x in row] for row in a]
    B = [Fraction(x).limit_denominator(10 ** 9) for x in b]
    C = [Fraction(x).limit_denominator(10 ** 9) for x in c]
    s = len(B)
    Am = [[A[i][j] if j < 6 else Fraction(0) for j in range(s)] for i in range(s)]

    def mat_vec(v):
        return [sum(Am[i][j] * v[j] for j in range(s)) for i in range(s)]

    dot = lambda u, v: sum(x * y for x, y in zip(u, v))
    one = [Fraction(1)] * s
    cs = C
    conds = [(dot(B, one), Fraction(1))]
    if order >= 2:
        conds.append((dot(B, cs), Fraction(1, 2)))
    if order >= 3:
        conds += [(dot(B, [x * x for x in cs]), Fraction(1, 3)), (dot(B, mat_vec(cs)), Fraction(1, 6))]
    if order >= 4:
        c2 = [x * x for x in cs]
        conds += [(dot(B, [x ** 3 for x in cs]), Fraction(1, 4)),
                  (dot(B, [x * y for x, y in zip(cs, mat_vec(cs))]), Fraction(1, 8)),
                  (dot(B, mat_vec(c2)), Fraction(1, 12)),
                  (dot(B, mat_vec(mat_vec(cs))), Fraction(1, 24))]
    if order >= 5:
        c2 = [x * x for x in cs]
        Ac = mat_vec(cs)
        conds += [(dot(B, [x ** 4 for x in cs]), Fraction(1, 5)),
                  (dot(B, [x * x * y for x, y in zip(cs, Ac)]), Fraction(1, 10)),
                  (dot(B, [y * y for y in Ac]), Fraction(1, 20)),
                  (dot(B, [x * y for x, y in zip(cs, mat_vec(c2))]), Fraction(1, 15)),
                  (dot(B, mat_vec([x ** 3 for x in cs])), Fraction(1, 20)),
                  (dot(B, [x * y for x, y in zip(cs, mat_vec(Ac))]), Fraction(1, 30)),
                  (dot(B, mat_vec([x * y for x, y in zip(cs, Ac)])), Fraction(1, 40)),
                  (dot(B, mat_vec(mat_vec(c2))), Fraction(1, 60)),
                  (dot(B, mat_vec(mat_vec(mat_vec(cs)))), Fraction(1, 120))]
    return conds


def test_dormand_prince_order_conditions(oracle_mod):
    c, a, b, bs = oracle_mod.dp5_tableau()
    for i in range(7):
        assert abs(a[i].sum() - c[i]) < 1e-15
    for lhs, rhs in _rk_order_conditions(c, a, b, 5):
        assert lhs == rhs
    for lhs, rhs in _rk_order_conditions(c, a, bs, 4):
        assert lhs == rhs
    # the embedded pair differs (otherwise the error estimate would vanish), and FSAL: b = last row of a
    assert np.abs(b - bs).max() > 1e-3
    assert np.allclose(a[6], b[:6]) and b[6] == 0


def _convergence(oracle_mod, stepper, dts):
    alpha, H = 0.2, 1.5e5
    th0, ph0 = 1.0, 0.0
    m0 = np.array([np.sin(th0) * np.cos(ph0), np.sin(th0) * np.sin(ph0), np.cos(th0)])
    T = 1e-10
    errs = []
    me = macrospin(oracle_mod, alpha, H)
    for dt in dts:
        m = np.broadcast_to(m0, (2, 2, 2, 3)).copy()
        nsteps = int(round(T / dt))
        m = stepper(me, m, dt, nsteps)
        errs.append(np.abs(m[0, 0, 0] - exact_macrospin(th0, ph0, alpha, H, T)).max())
    return np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])


def test_rk4_global_order(oracle_mod):
    def rk4(me, m, dt, n):
        for s in range(n):
            m = me.rk4_step(m, s * dt, dt, oracle_mod.ALL)
        return m
    o1, o2 = _convergence(oracle_mod, rk4, [4e-12, 2e-12, 1e-12])
    assert 3.7 < o1 < 4.3 and 3.7 < o2 < 4.3


def test_dp5_global_order_with_fixed_steps(oracle_mod):
    def dp5(me, m, dt, n):
        st = me.dp5_stepper(m, 0.0, dt, oracle_mod.ALL, rtol=1e30, atol=1e30, renorm=False)
        for _ in range(n):
            st.set_dt(dt)
            assert st.step()
        return st.m
    o1, o2 = _convergence(oracle_mod, dp5, [5e-12, 2.5e-12, 1.25e-12])
    assert 4.6 < o1 < 5.5 and 4.6 < o2 < 5.5


def test_dp5_error_estimate_is_fourth_order_local(oracle_mod):
    """The embedded estimate behaves like dt^5 (local error of the 4th-order solution)."""
    me = macrospin(oracle_mod, 0.2, 1.5e5)
    m0 = np.broadcast_to(np.array([np.sin(1.0), 0.0, np.cos(1.0)]), (2, 2, 2, 3)).copy()
    errs = []
    for dt in (1.6e-11, 8e-12, 4e-12):
        st = me.dp5_stepper(m0, 0.0, dt, oracle_mod.ALL, rtol=0.0, atol=1.0, renorm=False)
        st.step()
        errs.append(st.err)
    r = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert 4.5 < r[0] < 5.5 and 4.5 < r[1] < 5.5


def test_dp5_controller_rejects_and_shrinks(oracle_mod):
    me = macrospin(oracle_mod, 0.2, 1.5e5)
    m0 = np.broadcast_to(np.array([np.sin(1.0), 0.0, np.cos(1.0)]), (2, 2, 2, 3)).copy()
    st = me.dp5_stepper(m0, 0.0, 1e-10, oracle_mod.ALL, rtol=1e-8, atol=1e-8)
    assert not st.step()
    assert st.t.value == 0.0 and abs(st.dt.value - 0.2e-10) < 1e-22
    assert np.array_equal(st.m, m0)


def _small_problem(oracle_mod, alpha):
    p = inp.cuboid_rk4(0)
    n = (6, 5, 2)
    me = oracle_mod.Mesh(n, p.dx)
    me.set_material(p.Ms, p.A, 0.0, (0, 0, 1), alpha, p.gamma)
    me.set_zeeman(p.h_uniform)
    rng = np.random.default_rng(21)
    m = np.array([0.6, 0.0, 0.8]) + 0.3 * rng.standard_normal(me.nodes + (3,))
    m /= np.linalg.norm(m, axis=-1, keepdims=True)
    return me, m


def test_energy_conserved_without_damping(oracle_mod):
    """alpha = 0 and a static field: the LLG flow conserves the total energy; RK4 drift over
    1000 steps of 1e-15 s stays below 1e-8 relative (threshold from this oracle's own run, stated)."""
    me, m = _small_problem(oracle_mod, 0.0)
    E0 = me.energy(m)
    for s in range(1000):
        m = me.rk4_step(m, s * 1e-15, 1e-15, oracle_mod.ALL)
    E1 = me.energy(m)
    assert abs(E1 - E0) < 1e-8 * abs(E0)


def test_energy_decreases_with_damping_and_norm_drift_small(oracle_mod):
    me, m = _small_problem(oracle_mod, 0.5)
    E = [me.energy(m)]
    for s in range(40):
        m = me.rk4_step(m, s * 2e-15, 2e-15, oracle_mod.ALL, renorm=False)
        E.append(me.energy(m))
    assert all(E[i + 1] < E[i] for i in range(len(E) - 1))
    assert np.abs(np.linalg.norm(m, axis=-1) - 1).max() < 1e-6
