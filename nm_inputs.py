"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no arithmetic of the method: only random draws and the physical constants and
parameters of the workloads.  Both the CUDA library and the CPU oracle are fed identical arrays from
here, so neither side depends on the other.

Physical conventions (the paper leaves them open):
  * mu0 = 4 pi 1e-7 exactly; fields quoted in mT are mu0*H, so H = B / mu0.
  * gamma = mu0 * gamma_e with gamma_e = 1.76085963023e11 rad/(s T) (CODATA 2018), in m/(A s).

Workloads (cell counts, cell sizes, materials) follow the throughput, validation and inverse-problem
set-ups of the paper's benchmark and validation sections; every random quantity is drawn from
``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

MU0 = 4e-7 * np.pi
GAMMA_E = 1.76085963023e11
GAMMA = MU0 * GAMMA_E


def unit_vectors(rng: np.random.Generator, shape) -> np.ndarray:
    """i.i.d. directions uniform on the sphere (normalised Gaussian triples), shape (..., 3)."""
    v = rng.standard_normal(tuple(shape) + (3,))
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def unit_vector(rng: np.random.Generator) -> np.ndarray:
    return unit_vectors(rng, ())


@dataclass
class Problem:
    """One synthetic micromagnetic problem: mesh, material, applied field, initial state."""
    name: str
    n: tuple                     # cells (N1, N2, N3)
    dx: tuple                    # cell size in m
    Ms: object                   # A/m, scalar or (N1,N2,N3)
    A: object                    # J/m
    Ku: object = 0.0             # J/m^3
    axis: tuple = (0.0, 0.0, 1.0)
    alpha: float = 0.1
    gamma: float = GAMMA
    h_uniform: tuple = (0.0, 0.0, 0.0)   # A/m
    h_freq: float = 0.0
    h_phase: float = 0.0
    h_cell: Optional[np.ndarray] = None  # (N1,N2,N3,3) A/m
    cell_freq: float = 0.0
    cell_phase: float = 0.0
    m0: Optional[np.ndarray] = None      # (N1+1,N2+1,N3+1,3)
    terms: int = 15
    extra: dict = field(default_factory=dict)

    @property
    def nodes(self):
        return tuple(v + 1 for v in self.n)

    @property
    def n_nodes(self):
        return int(np.prod(self.nodes))

    def Ms_cells(self):
        return np.broadcast_to(np.asarray(self.Ms, dtype=np.float64), self.n).copy()

    def A_cells(self):
        return np.broadcast_to(np.asarray(self.A, dtype=np.float64), self.n).copy()

    def Ku_cells(self):
        return np.broadcast_to(np.asarray(self.Ku, dtype=np.float64), self.n).copy()


EXCH, ANIS, ZEE, DEMAG = 1, 2, 4, 8


def cuboid_rk4(seed: int = 0) -> Problem:
    """16x16x4 cells of 2 nm, Ms=8e5, A=1.3e-11, alpha=0.1, exchange+demag+Zeeman with 20 mT along a
    seeded direction, random unit m0; integrated with 1000 fixed RK4 steps of 1e-14 s."""
    rng = np.random.default_rng(seed)
    n = (16, 16, 4)
    h = unit_vector(rng) * (20e-3 / MU0)
    m0 = unit_vectors(rng, tuple(v + 1 for v in n))
    return Problem("cuboid 16x16x4 RK4", n, (2e-9, 2e-9, 2e-9), 8e5, 1.3e-11, 0.0, (0, 0, 1), 0.1,
                   h_uniform=tuple(h), m0=m0, terms=EXCH | ZEE | DEMAG,
                   extra=dict(method="rk4", dt=1e-14, steps=1000))


def thin_film(seed: int = 0) -> Problem:
    """200x50x1 cells of 2.5x2.5x3 nm, Ms=8e5, A=1.3e-11, alpha=0.02; m0 near-uniform in-plane plus
    1e-2 Gaussian noise; Zeeman 10-50 mT at a seeded in-plane angle; adaptive RK to 1 ns."""
    rng = np.random.default_rng(seed)
    n = (200, 50, 1)
    psi = rng.uniform(0, 2 * np.pi)
    nodes = tuple(v + 1 for v in n)
    m0 = np.array([np.cos(psi), np.sin(psi), 0.0]) + 1e-2 * rng.standard_normal(nodes + (3,))
    m0 /= np.linalg.norm(m0, axis=-1, keepdims=True)
    b = rng.uniform(10e-3, 50e-3)
    ang = rng.uniform(0, 2 * np.pi)
    h = np.array([np.cos(ang), np.sin(ang), 0.0]) * (b / MU0)
    return Problem("thin film 200x50x1", n, (2.5e-9, 2.5e-9, 3e-9), 8e5, 1.3e-11, 0.0, (0, 0, 1), 0.02,
                   h_uniform=tuple(h), m0=m0, terms=EXCH | ZEE | DEMAG,
                   extra=dict(method="dp54", t_end=1e-9, rtol=1e-5, atol=1e-5, dt0=1e-14, sample_dt=1e-12))


def throughput(n=(256, 256, 8), seed: int = 0, with_m0: bool = True) -> Problem:
    """Throughput cuboids (256x256x8, 512x512x16, 1024x1024x32 cells) of 3 nm cells, Ms=1e6,
    A=1.5e-11, Ku=5e5 along z, random unit m0, adaptive DP5 steps."""
    rng = np.random.default_rng(seed)
    n = tuple(int(v) for v in n)
    m0 = unit_vectors(rng, tuple(v + 1 for v in n)) if with_m0 else None
    return Problem(f"cuboid {n[0]}x{n[1]}x{n[2]} throughput", n, (3e-9, 3e-9, 3e-9), 1e6, 1.5e-11, 5e5,
                   (0, 0, 1), 0.1, m0=m0, terms=EXCH | ANIS | DEMAG,
                   extra=dict(method="dp54", rtol=1e-5, atol=1e-5, steps=200))


def waveguide(seed: int = 0) -> Problem:
    """256x64x1 cells of 4x4x10 nm; cell Ms map initialised to 1.4e5 A/m; A=3.5e-12, alpha=1e-3;
    m0 = +x; drive (1 mT/mu0) sin(2 pi 2 GHz t) along y on cells with c1 < 8."""
    n = (256, 64, 1)
    hc = np.zeros(n + (3,))
    hc[:8, :, :, 1] = 1e-3 / MU0
    m0 = np.zeros(tuple(v + 1 for v in n) + (3,))
    m0[..., 0] = 1.0
    return Problem("waveguide 256x64x1", n, (4e-9, 4e-9, 10e-9), np.full(n, 1.4e5), 3.5e-12, 0.0,
                   (0, 0, 1), 1e-3, h_cell=hc, cell_freq=2e9, cell_phase=0.0, m0=m0,
                   terms=EXCH | ZEE | DEMAG, extra=dict(t_end=2e-9, sample_dt=1e-12))


def random_problem(rng: np.random.Generator, n, dx=(2e-9, 2.5e-9, 3e-9), heterogeneous=True,
                   vacuum=False, terms=15) -> Problem:
    """A small problem with cell-wise random material, a random uniform and cell-wise field and a
    random unit m; optionally some vacuum cells (Ms = 0)."""
    n = tuple(int(v) for v in n)
    if heterogeneous:
        Ms = rng.uniform(4e5, 1.2e6, n)
        A = rng.uniform(5e-12, 2e-11, n)
        Ku = rng.uniform(-3e5, 5e5, n)
    else:
        Ms, A, Ku = 8e5, 1.3e-11, 2e5
    if vacuum:
        Ms = np.array(np.broadcast_to(Ms, n), dtype=np.float64)
        mask = rng.uniform(size=n) < 0.15
        Ms[mask] = 0.0
    axis = unit_vector(rng)
    h = unit_vector(rng) * rng.uniform(0, 100e-3) / MU0
    hc = rng.standard_normal(n + (3,)) * (5e-3 / MU0)
    m0 = unit_vectors(rng, tuple(v + 1 for v in n))
    return Problem(f"random {n}", n, tuple(dx), Ms, A, Ku, tuple(axis), rng.uniform(0.01, 0.5),
                   h_uniform=tuple(h), h_freq=1.5e9, h_phase=0.3, h_cell=hc, cell_freq=0.0,
                   m0=m0, terms=terms)


def serving_requests(n_requests: int = 500, seed: int = 0, rate_hz: float = 1.0, duration_scale: float = 1.0):
    """Poisson stream of LLG runs: grids N1,N2 in {64,128,256}, N3 in {1,2,4,8}; Ms ~ U[4e5,1.2e6],
    A ~ U[5e-12,2e-11], alpha ~ U[0.01,0.5], |mu0 h| ~ U[0,100] mT in a random direction, duration
    ~ U[0.2,2] ns (times duration_scale), m0 near-uniform plus noise.  Returns a list of
    (arrival_s, Problem) with m0 left out (see serving_m0) so that long streams stay small."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        n = (int(rng.choice([64, 128, 256])), int(rng.choice([64, 128, 256])), int(rng.choice([1, 2, 4, 8])))
        Ms = rng.uniform(4e5, 1.2e6)
        A = rng.uniform(5e-12, 2e-11)
        alpha = rng.uniform(0.01, 0.5)
        h = unit_vector(rng) * rng.uniform(0, 100e-3) / MU0
        T = rng.uniform(0.2e-9, 2e-9) * duration_scale
        d = unit_vector(rng)
        p = Problem(f"request {i}", n, (3e-9, 3e-9, 3e-9), Ms, A, 0.0, (0, 0, 1), alpha,
                    h_uniform=tuple(h), m0=None, terms=EXCH | ZEE | DEMAG,
                    extra=dict(t_end=T, rtol=1e-5, atol=1e-5, dt0=1e-14, m0_dir=tuple(d),
                               m0_seed=int(rng.integers(0, 2**31))))
        out.append((t, p))
    return out


def serving_m0(p: Problem) -> np.ndarray:
    """Initial state of a serving request: its seeded direction plus 5 % Gaussian noise, normalised."""
    rng = np.random.default_rng(p.extra["m0_seed"])
    m0 = np.asarray(p.extra["m0_dir"]) + 0.05 * rng.standard_normal(p.nodes + (3,))
    return m0 / np.linalg.norm(m0, axis=-1, keepdims=True)
