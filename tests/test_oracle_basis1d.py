"""Pins of the oracle's 1D nodal basis with full 3D integration (section "Low-Dimensional Geometries").

Closed forms that do not go through the 3D restriction the oracle uses: the lumped mass counts the
cells of a node's cross-section plane, a helix along the axis has the lumped-mass finite-element
Laplacian of a cosine wave inside and the one-sided difference at the ends, a uniform state has zero
exchange field and the textbook anisotropy and Zeeman fields, and a long wire of square cross-section
has the demagnetising factors of an infinite square prism (1/2 across, 0 along) at its centre.
"""
import numpy as np
import pytest

MU0 = 4e-7 * np.pi


@pytest.fixture(scope="module")
def b1():
    import oracle
    from oracle import basis1d
    return oracle, basis1d


def test_mass_counts_cells_of_the_plane(b1):
    oracle, basis1d = b1
    n, dx = (5, 3, 2), (2e-9, 3e-9, 1.5e-9)
    me = basis1d.Mesh1D(n, dx)
    Ms = 7e5
    me.set_material(Ms, 1e-11, 0.0, (0, 0, 1), 0.1, 2.2e5)
    mass = me.mass()
    assert mass.shape == (n[0] + 1, 1, 1)
    V = np.prod(dx)
    for i in range(n[0] + 1):
        cx = (i > 0) + (i < n[0])
        assert mass[i, 0, 0] == pytest.approx(MU0 * Ms * V / 2 * cx * n[1] * n[2], rel=1e-14)


@pytest.mark.parametrize("cross", [(1, 1), (2, 3)])
def test_axial_helix_exchange(b1, cross):
    """m = (cos kx, sin kx, 0): h_ex = -(2A/(mu0 Ms)) (2 - 2 cos k dx)/dx^2 m inside, and
    h_ex = (4A/(mu0 Ms dx^2)) (m_1 - m_0) at the first node."""
    oracle, basis1d = b1
    n, dx = (30, cross[0], cross[1]), (2e-9, 2.5e-9, 3e-9)
    me = basis1d.Mesh1D(n, dx)
    Ms, A = 8e5, 1.3e-11
    me.set_material(Ms, A, 0.0, (0, 0, 1), 0.1, 2.2e5)
    k = 2 * np.pi / (10 * dx[0])
    x = np.arange(n[0] + 1) * dx[0]
    m = np.zeros(me.nodes + (3,))
    m[:, 0, 0, 0] = np.cos(k * x)
    m[:, 0, 0, 1] = np.sin(k * x)
    h = me.h_eff(m, oracle.EXCH)[:, 0, 0]
    ref = -(2 * A / (MU0 * Ms)) * (2 - 2 * np.cos(k * dx[0])) / dx[0] ** 2 * m[:, 0, 0]
    scale = np.abs(ref).max()
    np.testing.assert_allclose(h[1:-1], ref[1:-1], rtol=1e-12, atol=1e-9 * scale)
    end = 4 * A / (MU0 * Ms * dx[0] ** 2) * (m[1, 0, 0] - m[0, 0, 0])
    np.testing.assert_allclose(h[0], end, rtol=1e-12, atol=1e-9 * scale)


def test_uniform_state_fields(b1):
    oracle, basis1d = b1
    n, dx = (6, 2, 3), (2e-9, 2e-9, 3e-9)
    me = basis1d.Mesh1D(n, dx)
    Ms, Ku = 6e5, 4e5
    e = np.array([0.3, -0.4, 0.8])
    e /= np.linalg.norm(e)
    me.set_material(Ms, 1.5e-11, Ku, tuple(e), 0.1, 2.2e5)
    hu = np.array([1e4, -2e4, 3e4])
    me.set_zeeman(tuple(hu))
    mu = np.array([0.6, 0.0, 0.8])
    m = np.broadcast_to(mu, me.nodes + (3,)).copy()
    assert np.abs(me.h_eff(m, oracle.EXCH)).max() <= 1e-6
    h_an = me.h_eff(m, oracle.ANIS)
    np.testing.assert_allclose(h_an, np.broadcast_to(2 * Ku / (MU0 * Ms) * (mu @ e) * e, h_an.shape), rtol=1e-12)
    h_z = me.h_eff(m, oracle.ZEE)
    np.testing.assert_allclose(h_z, np.broadcast_to(hu, h_z.shape), rtol=1e-13)


def test_long_square_wire_demag(b1):
    """A 200-cell wire of one 2 nm cell cross-section: at its centre the demagnetising factor across the
    wire is that of an infinite square prism, 1/2, and the one along it vanishes (both within the end
    corrections, O((w/L)^2))."""
    oracle, basis1d = b1
    n, dx = (200, 1, 1), (2e-9, 2e-9, 2e-9)
    me = basis1d.Mesh1D(n, dx)
    Ms = 8e5
    me.set_material(Ms, 1e-11, 0.0, (0, 0, 1), 0.1, 2.2e5)
    c = n[0] // 2
    m = np.zeros(me.nodes + (3,))
    m[..., 1] = 1.0
    h = me.h_eff(m, oracle.DEMAG)[c, 0, 0]
    assert abs(h[1] / -Ms - 0.5) < 1e-4
    assert abs(h[0]) < 1e-9 * Ms and abs(h[2]) < 1e-9 * Ms
    m[..., 1] = 0.0
    m[..., 0] = 1.0
    h = me.h_eff(m, oracle.DEMAG)[c, 0, 0]
    assert 0.0 < h[0] / -Ms < 1e-4
    assert abs(h[1]) < 1e-9 * Ms and abs(h[2]) < 1e-9 * Ms
