"""Pins of the oracle's local field terms (exchange, uniaxial anisotropy, Zeeman) and lumped mass.

Every expected value here comes from the paper (the printed coefficient of the generated exchange
code, Lst. "lst:form_code"), from closed forms derived by hand, or from invariants; none comes from
the oracle itself or from the CUDA path.
"""
import os

import numpy as np
import pytest

import nm_inputs as inp

MU0 = 4e-7 * np.pi
HERE = os.path.dirname(os.path.abspath(__file__))


def _golden_lst2():
    with open(os.path.join(HERE, "golden", "lst2_exchange_coefficient.txt")) as f:
        for line in f:
            if line.startswith("coefficient"):
                return float(line.split()[1])
    raise RuntimeError("coefficient missing")


def _mesh(oracle_mod, n, dx, Ms=8e5, A=1.3e-11, Ku=0.0, axis=(0, 0, 1), alpha=0.1, gamma=inp.GAMMA):
    me = oracle_mod.Mesh(n, dx)
    me.set_material(Ms, A, Ku, axis, alpha, gamma)
    return me


# ---------------------------------------------------------------------------------- basis (Eq. nodal_basis)
def test_basis_kronecker_and_partition_of_unity(oracle_mod):
    rng = np.random.default_rng(1)
    for li in range(8):
        for lj in range(8):
            v = ((lj >> 2) & 1, (lj >> 1) & 1, lj & 1)
            assert oracle_mod.phi(li, *v) == (1.0 if li == lj else 0.0)
    for _ in range(20):
        x = rng.uniform(0, 1, 3)
        assert abs(sum(oracle_mod.phi(li, *x) for li in range(8)) - 1.0) < 1e-15


# ---------------------------------------------------------------------------------- element matrices
@pytest.mark.parametrize("dx", [(1.0, 1.0, 1.0), (2e-9, 3e-9, 5e-9), (2.5e-9, 2.5e-9, 3e-9), (4e-9, 4e-9, 10e-9)])
def test_exchange_diagonal_matches_listing_coefficient(oracle_mod, dx):
    """Lst. "lst:form_code" prints 0.222222222222222 * (dx0 dx1/dx2 + dx0 dx2/dx1 + dx1 dx2/dx0) as the
    self-coupling of the exchange element matrix; exact (Gauss) integration gives 2/9."""
    c = _golden_lst2()
    K, M, Phi = oracle_mod.element_matrices(dx)
    expect = c * (dx[0] * dx[1] / dx[2] + dx[0] * dx[2] / dx[1] + dx[1] * dx[2] / dx[0])
    assert np.allclose(np.diag(K), expect, rtol=1e-14, atol=0)
    # the printed coefficient carries 15 digits; it is 2/9
    assert abs(c - 2.0 / 9.0) < 5e-16
    # rows of the stiffness sum to zero (constants are in the kernel), the mass rows to V/8
    V = np.prod(dx)
    assert np.abs(K.sum(1)).max() < 1e-13 * np.abs(K).max()
    assert np.allclose(M.sum(1), V / 8, rtol=1e-14)
    assert np.allclose(Phi, V / 8, rtol=1e-14)
    # 1D closed forms: M = prod (h/6)[[2,1],[1,2]], e.g. the (0,7) corner entry is V/216
    assert abs(M[0, 7] - V / 216) < 1e-14 * V


# ---------------------------------------------------------------------------------- mass lumping (Eq. mass_lumping)
def test_lumped_mass_counts_adjacent_cells(oracle_mod):
    n, dx, Ms = (4, 3, 2), (2e-9, 3e-9, 4e-9), 7e5
    me = _mesh(oracle_mod, n, dx, Ms=Ms)
    mass = me.mass()
    V = np.prod(dx)
    for idx in np.ndindex(*me.nodes):
        cnt = 1
        for k in range(3):
            cnt *= 1 if idx[k] in (0, n[k]) else 2
        assert abs(mass[idx] - MU0 * Ms * V / 8 * cnt) < 1e-14 * MU0 * Ms * V


def test_lumped_mass_heterogeneous(oracle_mod):
    rng = np.random.default_rng(2)
    n, dx = (3, 2, 2), (2e-9, 2e-9, 2e-9)
    Ms = rng.uniform(1e5, 1e6, n)
    me = _mesh(oracle_mod, n, dx, Ms=Ms)
    mass = me.mass()
    V = np.prod(dx)
    for idx in np.ndindex(*me.nodes):
        s = 0.0
        for c in np.ndindex(2, 2, 2):
            cc = tuple(idx[k] - c[k] for k in range(3))
            if all(0 <= cc[k] < n[k] for k in range(3)):
                s += Ms[cc]
        assert abs(mass[idx] - MU0 * V / 8 * s) < 1e-13 * MU0 * V * 1e6


# ---------------------------------------------------------------------------------- exchange
def test_exchange_uniform_m_gives_zero(oracle_mod):
    rng = np.random.default_rng(3)
    n = (5, 4, 3)
    me = _mesh(oracle_mod, n, (2e-9, 2.5e-9, 3e-9), Ms=rng.uniform(4e5, 1e6, n), A=rng.uniform(5e-12, 2e-11, n))
    m = np.broadcast_to(inp.unit_vector(rng), me.nodes + (3,)).copy()
    h = me.h_eff(m, oracle_mod.EXCH)
    assert np.abs(h).max() < 1e-6  # A/m, against fields of order 1e6 for non-uniform m
    assert abs(me.energy(m, oracle_mod.EXCH)) < 1e-35


@pytest.mark.parametrize("k_cells", [0.3, 1.1])
def test_exchange_helix_energy_and_field(oracle_mod, k_cells):
    """m_n = (cos k x_n, sin k x_n, 0): the trilinear interpolant has |d m/dx|^2 = (2 - 2 cos k dx)/dx^2
    on every cell, so E = A V_tot (2 - 2cos k dx)/dx^2 exactly; the lumped field is
    -(2A/(mu0 Ms)) (2 - 2 cos k dx)/dx^2 m_n inside and (4A/(mu0 Ms dx^2))(m_1 - m_0) on the x faces."""
    n, dx = (9, 3, 2), (2e-9, 3e-9, 2.5e-9)
    A, Ms = 1.3e-11, 8e5
    me = _mesh(oracle_mod, n, dx, Ms=Ms, A=A)
    k = k_cells / dx[0]
    x = np.arange(n[0] + 1) * dx[0]
    m = np.zeros(me.nodes + (3,))
    m[..., 0] = np.cos(k * x)[:, None, None]
    m[..., 1] = np.sin(k * x)[:, None, None]
    Vtot = np.prod(n) * np.prod(dx)
    g = (2 - 2 * np.cos(k * dx[0])) / dx[0] ** 2
    E = me.energy(m, oracle_mod.EXCH)
    assert abs(E - A * Vtot * g) < 1e-12 * A * Vtot * g
    h = me.h_eff(m, oracle_mod.EXCH)
    inner = -(2 * A / (MU0 * Ms)) * g * m[1:-1]
    assert np.abs(h[1:-1] - inner).max() < 1e-9 * np.abs(inner).max()
    left = 4 * A / (MU0 * Ms * dx[0] ** 2) * (m[1] - m[0])
    right = 4 * A / (MU0 * Ms * dx[0] ** 2) * (m[-2] - m[-1])
    assert np.abs(h[0] - left).max() < 1e-9 * np.abs(left).max()
    assert np.abs(h[-1] - right).max() < 1e-9 * np.abs(right).max()


def test_exchange_jump_condition_two_phase(oracle_mod):
    """Eq. exchange_jump: with A1 on the left and A2 on the right half, a profile that is piecewise
    linear in x with slopes satisfying A1 s1 = A2 s2 is an exchange equilibrium at every inner node,
    including the interface node; equal slopes are not."""
    n, dx = (8, 2, 2), (2e-9, 2e-9, 2e-9)
    A1, A2 = 1.0e-11, 2.5e-11
    A = np.full(n, A1)
    A[n[0] // 2:] = A2
    me = _mesh(oracle_mod, n, dx, Ms=8e5, A=A)
    x = np.arange(n[0] + 1) * dx[0]
    xi = x[n[0] // 2]
    for s2, expect_zero in ((A1 / A2, True), (1.0, False)):
        u = np.where(x <= xi, x - xi, s2 * (x - xi)) * 1e7
        m = np.zeros(me.nodes + (3,))
        m[..., 0] = 1.0
        m[..., 1] = u[:, None, None]
        h = me.h_eff(m, oracle_mod.EXCH)
        iface = np.abs(h[n[0] // 2]).max()
        inner = np.abs(h[1:-1]).max()
        scale = 2 * A2 / (MU0 * 8e5) * 1e7 / dx[0]
        if expect_zero:
            assert inner < 1e-9 * scale
        else:
            assert iface > 1e-2 * scale


# ---------------------------------------------------------------------------------- anisotropy and Zeeman
def test_anisotropy_uniform_m(oracle_mod):
    """E = -int Ku (m.e)^2: for uniform m the consistent-mass rows sum to V/8, so every node (boundary
    included) gets H = 2 Ku/(mu0 Ms) (m.e) e."""
    rng = np.random.default_rng(4)
    Ku, Ms = 4e5, 9e5
    e = inp.unit_vector(rng)
    me = _mesh(oracle_mod, (4, 3, 2), (2e-9, 3e-9, 4e-9), Ms=Ms, Ku=Ku, axis=e)
    mu = inp.unit_vector(rng)
    m = np.broadcast_to(mu, me.nodes + (3,)).copy()
    h = me.h_eff(m, oracle_mod.ANIS)
    expect = 2 * Ku / (MU0 * Ms) * np.dot(mu, e) * e
    assert np.abs(h - expect).max() < 1e-12 * np.abs(expect).max()
    E = me.energy(m, oracle_mod.ANIS)
    Vtot = 4 * 3 * 2 * 2e-9 * 3e-9 * 4e-9
    assert abs(E + Ku * np.dot(mu, e) ** 2 * Vtot) < 1e-12 * Ku * Vtot


def test_zeeman_uniform_and_time_dependent(oracle_mod):
    rng = np.random.default_rng(5)
    n = (3, 3, 2)
    me = _mesh(oracle_mod, n, (2e-9, 2e-9, 2e-9), Ms=rng.uniform(3e5, 1e6, n))
    hu = inp.unit_vector(rng) * 3e4
    me.set_zeeman(hu, freq=2e9, phase=0.4)
    m = inp.unit_vectors(rng, me.nodes)
    t = 1.3e-10
    h = me.h_eff(m, oracle_mod.ZEE, t)
    expect = hu * np.sin(2 * np.pi * 2e9 * t + 0.4)
    assert np.abs(h - expect).max() < 1e-12 * np.abs(hu).max()
    # a cell-wise field is averaged with Ms weights over the adjacent cells
    hc = rng.standard_normal(n + (3,)) * 1e4
    Ms = rng.uniform(3e5, 1e6, n)
    me.set_material(Ms, 1e-11, 0, (0, 0, 1), 0.1, inp.GAMMA)
    me.set_zeeman((0, 0, 0), h_cell=hc)
    h = me.h_eff(m, oracle_mod.ZEE)
    node = (1, 2, 1)
    num, den = np.zeros(3), 0.0
    for c in np.ndindex(2, 2, 2):
        cc = tuple(node[k] - c[k] for k in range(3))
        if all(0 <= cc[k] < n[k] for k in range(3)):
            num += Ms[cc] * hc[cc]
            den += Ms[cc]
    assert np.abs(h[node] - num / den).max() < 1e-12 * np.abs(num / den).max()


# ---------------------------------------------------------------------------------- variational consistency
@pytest.mark.parametrize("vacuum", [False, True])
def test_field_is_minus_energy_gradient_over_mass(oracle_mod, vacuum):
    """H_n = -(1/mass_n) dE/dm_n for every term (Eqs. heff, weak_form, mass_lumping).  The energies
    are quadratic in m, so a central difference with a unit step is exact up to rounding."""
    rng = np.random.default_rng(6 + vacuum)
    p = inp.random_problem(rng, (3, 3, 2), vacuum=vacuum)
    me = oracle_mod.Mesh(p.n, p.dx)
    me.set_material(p.Ms_cells(), p.A_cells(), p.Ku_cells(), p.axis, p.alpha, p.gamma)
    me.set_zeeman(p.h_uniform, p.h_freq, p.h_phase, p.h_cell)
    m = p.m0
    mass = me.mass()
    t = 2e-10
    for terms in (oracle_mod.EXCH, oracle_mod.ANIS, oracle_mod.ZEE, oracle_mod.DEMAG, oracle_mod.ALL):
        h = me.h_eff(m, terms, t)
        scale = np.abs(h).max()
        for idx in [(0, 0, 0, 0), (1, 1, 1, 2), (3, 3, 2, 1), (2, 1, 0, 1), (1, 2, 2, 0)]:
            if mass[idx[:3]] == 0.0:
                assert h[idx] == 0.0
                continue
            mp_, mm_ = m.copy(), m.copy()
            mp_[idx] += 0.5
            mm_[idx] -= 0.5
            dE = me.energy(mp_, terms, t) - me.energy(mm_, terms, t)
            assert abs(-dE / mass[idx[:3]] - h[idx]) < 1e-9 * scale, (terms, idx)


def test_linear_terms_are_symmetric(oracle_mod):
    """<u, dE_lin(v)> = <v, dE_lin(u)> for exchange, anisotropy and demag (a symmetric bilinear energy)."""
    rng = np.random.default_rng(8)
    p = inp.random_problem(rng, (4, 3, 2))
    me = oracle_mod.Mesh(p.n, p.dx)
    me.set_material(p.Ms_cells(), p.A_cells(), p.Ku_cells(), p.axis, p.alpha, p.gamma)
    u = rng.standard_normal(me.nodes + (3,))
    v = rng.standard_normal(me.nodes + (3,))
    for terms in (oracle_mod.EXCH, oracle_mod.ANIS, oracle_mod.DEMAG):
        a = np.sum(u * me.variation(v, terms))
        b = np.sum(v * me.variation(u, terms))
        assert abs(a - b) < 1e-12 * max(abs(a), abs(b), 1e-300), terms
