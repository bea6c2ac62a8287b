"""Pins of the oracle's demagnetisation field (Sec. "Demagnetization Field": FFT-ready cuboid-cell
tensor with node->cell and cell->node averaging; the oracle sums directly).

Independent references: Aharoni's closed form for the demagnetising factors of a rectangular prism
(A. Aharoni, J. Appl. Phys. 83, 3432 (1998)), the point-dipole far field, the trace identities of
the magnetostatic tensor, and the cube.
"""
import math

import numpy as np
import pytest

import nm_inputs as inp
from helpers import aharoni_Dz, aharoni_factors


def test_aharoni_reference_is_consistent():
    assert abs(aharoni_Dz(1, 1, 1) - 1 / 3) < 1e-14
    for L in [(1, 2, 3), (5, 1, 0.3), (2.5, 2.5, 3)]:
        assert abs(aharoni_factors(L).sum() - 1) < 1e-13


def test_cube_self_term(oracle_mod):
    N = oracle_mod.newell((1.0, 1.0, 1.0), (0, 0, 0))
    assert np.allclose(N[:3], 1 / 3, rtol=0, atol=1e-15)
    assert np.abs(N[3:]).max() < 1e-15


@pytest.mark.parametrize("dx", [(1, 2, 3), (2.5e-9, 2.5e-9, 3e-9), (4e-9, 4e-9, 10e-9), (3, 0.5, 1.7)])
def test_self_term_equals_prism_factors(oracle_mod, dx):
    N = oracle_mod.newell(dx, (0, 0, 0))
    assert np.allclose(N[:3], aharoni_factors(dx), rtol=1e-13, atol=1e-15)
    assert abs(N[:3].sum() - 1) < 1e-14
    assert np.abs(N[3:]).max() < 1e-15


def test_trace_vanishes_off_self(oracle_mod):
    rng = np.random.default_rng(11)
    dx = (2e-9, 3e-9, 2.5e-9)
    for _ in range(20):
        c = rng.integers(-6, 7, 3)
        if not c.any():
            continue
        N = oracle_mod.newell(dx, c * np.array(dx))
        assert abs(N[:3].sum()) < 1e-14 * max(1.0, np.abs(N).max()) + 1e-17


def test_far_field_is_point_dipole(oracle_mod):
    """N(r) -> -(V/4 pi) (3 r r^T/r^2 - I)/r^3 with a relative error of order (dx/r)^2."""
    dx = np.array([2e-9, 3e-9, 2.5e-9])
    V = dx.prod()
    d = np.array([0.6, -0.7, 0.4])
    d /= np.linalg.norm(d)
    errs = []
    for R in (20e-9, 40e-9, 80e-9):
        c = np.round(d * R / dx)
        r = c * dx
        rn = np.linalg.norm(r)
        D = -(V / (4 * np.pi)) * (3 * np.outer(r, r) / rn ** 2 - np.eye(3)) / rn ** 3
        N = oracle_mod.newell(dx, r)
        Nm = np.array([[N[0], N[3], N[4]], [N[3], N[1], N[5]], [N[4], N[5], N[2]]])
        errs.append(np.abs(Nm - D).max() / np.abs(D).max())
    assert errs[-1] < 2e-3
    # error falls with the square of the distance (ratio ~4 per doubling)
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def test_tensor_parity(oracle_mod):
    dx = (2e-9, 3e-9, 2.5e-9)
    a = oracle_mod.newell(dx, (4e-9, 6e-9, 5e-9))
    b = oracle_mod.newell(dx, (-4e-9, 6e-9, 5e-9))
    c = oracle_mod.newell(dx, (4e-9, -6e-9, -5e-9))
    assert np.allclose(b, a * np.array([1, 1, 1, -1, -1, 1]), rtol=1e-13)
    assert np.allclose(c, a * np.array([1, 1, 1, -1, -1, 1]), rtol=1e-13)


@pytest.mark.parametrize("n", [(3, 2, 2), (4, 3, 1), (2, 2, 3)])
def test_block_sum_is_prism_factor(oracle_mod, n):
    """(1/Nc) sum_{c,c'} N(c-c') is the demag tensor of the whole prism: checked against the same
    formula for one big cell and against Aharoni's closed form."""
    dx = (2e-9, 3e-9, 2.5e-9)
    me = oracle_mod.Mesh(n, dx)
    T = me.tensor()
    sgn = np.array([1, 1, 1])
    S = np.zeros(6)
    for c in np.ndindex(*n):
        for b in np.ndindex(*n):
            e = np.array(c) - np.array(b)
            t = T[tuple(np.abs(e))]
            s = np.where(e < 0, -1, 1) * sgn
            S += t * np.array([1, 1, 1, s[0] * s[1], s[0] * s[2], s[1] * s[2]])
    S /= np.prod(n)
    L = np.array(n) * np.array(dx)
    big = oracle_mod.newell(L, (0, 0, 0))
    assert np.allclose(S, big, rtol=0, atol=1e-14)
    assert np.allclose(S[:3], aharoni_factors(L), rtol=1e-12)


def test_uniform_m_mean_field_is_prism_field(oracle_mod):
    """For uniform m in a full cuboid, the volume-averaged cell field is -N_prism Ms m, and the node
    field of a single cube is -Ms m/3 on all eight nodes."""
    rng = np.random.default_rng(12)
    n, dx, Ms = (5, 3, 2), (2e-9, 2.5e-9, 3e-9), 8e5
    me = oracle_mod.Mesh(n, dx)
    me.set_material(Ms, 0.0, 0.0, (0, 0, 1), 0.1, inp.GAMMA)
    mu = inp.unit_vector(rng)
    m = np.broadcast_to(mu, me.nodes + (3,)).copy()
    Hc = me.demag_cells(m)
    D = aharoni_factors(np.array(n) * np.array(dx))
    assert np.allclose(Hc.reshape(-1, 3).mean(0), -Ms * D * mu, rtol=1e-11, atol=1e-9)
    cube = oracle_mod.Mesh((1, 1, 1), (3e-9, 3e-9, 3e-9))
    cube.set_material(Ms, 0.0, 0.0, (0, 0, 1), 0.1, inp.GAMMA)
    m1 = np.broadcast_to(mu, (2, 2, 2, 3)).copy()
    h = cube.h_eff(m1, oracle_mod.DEMAG)
    assert np.allclose(h, -Ms * mu / 3, rtol=0, atol=1e-9 * Ms)


def test_thin_film_limit(oracle_mod):
    """A wide film magnetised along its normal has an interior field close to -Ms m_z."""
    n, dx, Ms = (40, 40, 1), (3e-9, 3e-9, 1e-9), 8e5
    me = oracle_mod.Mesh(n, dx)
    me.set_material(Ms, 0.0, 0.0, (0, 0, 1), 0.1, inp.GAMMA)
    m = np.zeros(me.nodes + (3,))
    m[..., 2] = 1.0
    h = me.h_eff(m, oracle_mod.DEMAG)
    hz = h[20, 20, 0, 2] / -Ms
    # 1 - O(t/L): for t/L = 1/120 the deficit is below a few percent
    assert 0.97 < hz < 1.0
    assert abs(h[20, 20, 0, 0]) < 1e-9 * Ms and abs(h[20, 20, 0, 1]) < 1e-9 * Ms


def test_results_do_not_depend_on_the_thread_count(oracle_mod):
    """The direct-sum field and the tensor are bitwise the same on one host thread and on all of them
    (the CPU baseline is timed both ways)."""
    rng = np.random.default_rng(12)
    p = inp.random_problem(rng, (6, 5, 3))
    me = oracle_mod.Mesh(p.n, p.dx)
    me.set_material(p.Ms_cells(), p.A_cells(), p.Ku_cells(), p.axis, p.alpha, p.gamma)
    all_threads = oracle_mod.num_threads()
    h_all = me.h_eff(p.m0, oracle_mod.DEMAG)
    try:
        oracle_mod.set_num_threads(1)
        assert oracle_mod.num_threads() == 1
        me1 = oracle_mod.Mesh(p.n, p.dx)
        me1.set_material(p.Ms_cells(), p.A_cells(), p.Ku_cells(), p.axis, p.alpha, p.gamma)
        h_one = me1.h_eff(p.m0, oracle_mod.DEMAG)
    finally:
        oracle_mod.set_num_threads(all_threads)
    assert np.array_equal(h_all, h_one)
