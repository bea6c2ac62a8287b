"""Pins of the oracle's interfacial DMI term (a reading: the paper lists antisymmetric exchange among the
energies its scheme handles, section "Nodal Finite-Difference Scheme", without giving the energy; here
E = int D [m_z div m - (m . grad) m_z], interface normal along z).

The variation is checked against brute-force central differences of the energy (which is evaluated by
quadrature of the nodal interpolant, not through the element matrices), the operator against its
symmetry, and the energy of a Neel spiral against the continuum value -D k V.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def oracle():
    import oracle as o
    return o


def _mesh(o, n=(4, 3, 2), dx=(2e-9, 2.5e-9, 1.5e-9), D=None, seed=0):
    rng = np.random.default_rng(seed)
    me = o.Mesh(n, dx)
    Ms = rng.uniform(5e5, 1e6, n)
    me.set_material(Ms, 1e-11, 0.0, (0, 0, 1), 0.1, 2.2e5)
    me.set_dmi(rng.uniform(-3e-3, 3e-3, n) if D is None else D)
    return me, rng


def test_variation_is_the_energy_gradient(oracle):
    me, rng = _mesh(oracle)
    m = rng.standard_normal(me.nodes + (3,))
    dE = me.variation(m, oracle.DMI)
    eps = 1e-6
    for _ in range(6):
        idx = tuple(rng.integers(0, s) for s in me.nodes) + (int(rng.integers(0, 3)),)
        mp, mm = m.copy(), m.copy()
        mp[idx] += eps
        mm[idx] -= eps
        fd = (me.energy(mp, oracle.DMI) - me.energy(mm, oracle.DMI)) / (2 * eps)
        assert dE[idx] == pytest.approx(fd, rel=1e-7, abs=1e-9 * np.abs(dE).max())


def test_operator_is_symmetric(oracle):
    me, rng = _mesh(oracle, seed=1)
    v = rng.standard_normal(me.nodes + (3,))
    w = rng.standard_normal(me.nodes + (3,))
    a = np.sum(v * me.variation(w, oracle.DMI))
    b = np.sum(w * me.variation(v, oracle.DMI))
    assert a == pytest.approx(b, rel=1e-12)
    # the energy is the quadratic form of that operator: E(m) = <m, dE(m)> / 2
    assert me.energy(v, oracle.DMI) == pytest.approx(0.5 * np.sum(v * me.variation(v, oracle.DMI)), rel=1e-12)


@pytest.mark.parametrize("sign", [1, -1])
def test_neel_spiral_energy(oracle, sign):
    """m = (cos kx, 0, sin kx): continuum density D [m_z dx m_x - m_x dx m_z] = -D k; the interpolant's
    energy agrees to O((k dx)^2) and flips with the chirality."""
    n, dx = (48, 2, 1), (1e-9, 2e-9, 2e-9)
    me = oracle.Mesh(n, dx)
    me.set_material(8e5, 1e-11, 0.0, (0, 0, 1), 0.1, 2.2e5)
    D = 2e-3
    me.set_dmi(D)
    k = sign * 2 * np.pi / (16 * dx[0])
    x = np.arange(n[0] + 1) * dx[0]
    m = np.zeros(me.nodes + (3,))
    m[..., 0] = np.cos(k * x)[:, None, None]
    m[..., 2] = np.sin(k * x)[:, None, None]
    V = np.prod(n) * np.prod(dx)
    E = me.energy(m, oracle.DMI)
    ref = -D * k * V
    assert abs(E - ref) <= 0.05 * abs(ref)
    # the finite-element value: exact derivative of the linear interpolant, sin(k dx)/(k dx) of the continuum
    assert E == pytest.approx(ref * np.sin(k * dx[0]) / (k * dx[0]), rel=1e-10)


def test_uniform_state_interior_field_vanishes(oracle):
    """For uniform m the DMI variation cancels at interior nodes (translation invariance) and only the
    boundary nodes feel the term."""
    n = (6, 5, 3)
    me, _ = _mesh(oracle, n=n, D=1.5e-3)
    m = np.broadcast_to(np.array([0.6, 0.0, 0.8]), me.nodes + (3,)).copy()
    dE = me.variation(m, oracle.DMI)
    assert np.abs(dE[1:-1, 1:-1, :]).max() <= 1e-12 * np.abs(dE).max()
    assert np.abs(dE).max() > 0
