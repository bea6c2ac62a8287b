"""Pins of the oracle's 2D nodal basis with full 3D integration (section "Low-Dimensional Geometries").

Closed forms that do not go through the 3D restriction the oracle uses: the lumped mass counts the
cells of a node column, an in-plane helix has the lumped-mass finite-element Laplacian of a cosine wave,
a uniform state has zero exchange field and the textbook anisotropy and Zeeman fields, and a wide film
magnetised out of plane has a demag field close to -Ms at its centre.
"""
import numpy as np
import pytest

MU0 = 4e-7 * np.pi


@pytest.fixture(scope="module")
def b2():
    import oracle
    from oracle import basis2d
    return oracle, basis2d


def test_mass_counts_cells_of_the_column(b2):
    oracle, basis2d = b2
    n, dx = (4, 3, 2), (2e-9, 3e-9, 1.5e-9)
    me = basis2d.Mesh2D(n, dx)
    Ms = 7e5
    me.set_material(Ms, 1e-11, 0.0, (0, 0, 1), 0.1, 2.2e5)
    mass = me.mass()[..., 0]
    V = np.prod(dx)
    for i in range(n[0] + 1):
        for j in range(n[1] + 1):
            cx = (i > 0) + (i < n[0])
            cy = (j > 0) + (j < n[1])
            assert mass[i, j] == pytest.approx(MU0 * Ms * V / 4 * cx * cy * n[2], rel=1e-14)


@pytest.mark.parametrize("n3", [1, 3])
def test_inplane_helix_exchange(b2, n3):
    """m = (cos kx, sin kx, 0): h_ex = -(2A/(mu0 Ms)) (2 - 2 cos k dx)/dx^2 m at nodes away from the x ends."""
    oracle, basis2d = b2
    n, dx = (24, 3, n3), (2e-9, 2.5e-9, 3e-9)
    me = basis2d.Mesh2D(n, dx)
    Ms, A = 8e5, 1.3e-11
    me.set_material(Ms, A, 0.0, (0, 0, 1), 0.1, 2.2e5)
    k = 2 * np.pi / (12 * dx[0])
    x = np.arange(n[0] + 1) * dx[0]
    m = np.zeros(me.nodes + (3,))
    m[..., 0] = np.cos(k * x)[:, None, None]
    m[..., 1] = np.sin(k * x)[:, None, None]
    h = me.h_eff(m, oracle.EXCH)
    ref = -(2 * A / (MU0 * Ms)) * (2 - 2 * np.cos(k * dx[0])) / dx[0] ** 2 * m
    np.testing.assert_allclose(h[1:-1], ref[1:-1], rtol=1e-12, atol=1e-9 * np.abs(ref).max())


def test_uniform_state_fields(b2):
    oracle, basis2d = b2
    n, dx = (5, 4, 2), (2e-9, 2e-9, 3e-9)
    me = basis2d.Mesh2D(n, dx)
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


def test_wide_film_out_of_plane_demag(b2):
    """A 40x40 film, 1 nm thick on 2 nm cells, magnetised along z: H_z close to -Ms at the centre."""
    oracle, basis2d = b2
    n, dx = (40, 40, 1), (2e-9, 2e-9, 1e-9)
    me = basis2d.Mesh2D(n, dx)
    Ms = 8e5
    me.set_material(Ms, 1e-11, 0.0, (0, 0, 1), 0.1, 2.2e5)
    m = np.zeros(me.nodes + (3,))
    m[..., 2] = 1.0
    h = me.h_eff(m, oracle.DEMAG)
    c = n[0] // 2
    assert -1.0 < h[c, c, 0, 2] / Ms < -0.95
    assert abs(h[c, c, 0, 0]) < 1e-6 * Ms and abs(h[c, c, 0, 1]) < 1e-6 * Ms
