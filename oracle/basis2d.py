"""Two-dimensional nodal basis with full three-dimensional integration (section "Low-Dimensional
Geometries" of the paper) for the FP64 oracle.

TEST INFRASTRUCTURE ONLY, under the same rule as the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it.  It never imports the
CUDA library.

The 2D basis function of node (i1, i2) is constant along the third axis over all N3 cell layers; it is
the sum of the 3D nodal basis functions of the node column (i1, i2, 0..N3), which form a partition of
unity along z.  The 2D Galerkin system is therefore the 3D one restricted to magnetisations that are
constant along z: with m3(i1, i2, k) = m2(i1, i2),

    dE/dm2_n = sum_k dE/dm3_(n,k)        (chain rule)
    mass2_n  = mu0 int Ms phi2_n = sum_k mass3_(n,k)
    h2_n     = -dE/dm2_n / mass2_n

and the LLG right-hand side and the integrators act on the (N1+1) x (N2+1) x 1 nodal field.  This module
evaluates exactly that, on top of the 3D oracle.
"""
from __future__ import annotations

import numpy as np

from . import ALL, Mesh


class Mesh2D:
    """N1 x N2 x N3 cells, nodal 2D basis: nodes (N1+1, N2+1, 1)."""

    def __init__(self, n, dx):
        self.m3 = Mesh(n, dx)
        self.n = self.m3.n
        self.cells = self.m3.cells
        self.nodes = (self.n[0] + 1, self.n[1] + 1, 1)

    def set_material(self, *args, **kw):
        self.m3.set_material(*args, **kw)
        self.alpha, self.gamma = self.m3.alpha, self.m3.gamma

    def set_zeeman(self, *args, **kw):
        self.m3.set_zeeman(*args, **kw)

    def lift(self, m2):
        m2 = np.asarray(m2, dtype=np.float64).reshape(self.nodes + (3,))
        return np.repeat(m2, self.n[2] + 1, axis=2)

    def mass(self) -> np.ndarray:
        return self.m3.mass().sum(axis=2, keepdims=True)

    def variation(self, m2, terms=ALL, t=0.0) -> np.ndarray:
        return self.m3.variation(self.lift(m2), terms, t).sum(axis=2, keepdims=True)

    def h_eff(self, m2, terms=ALL, t=0.0) -> np.ndarray:
        mass = self.mass()[..., None]
        dE = self.variation(m2, terms, t)
        return np.where(mass > 0.0, -dE / np.where(mass > 0.0, mass, 1.0), 0.0)

    def llg_rhs(self, m2, terms=ALL, t=0.0) -> np.ndarray:
        """Eq. llg per node, zero on nodes without magnetic material."""
        m2 = np.asarray(m2, dtype=np.float64).reshape(self.nodes + (3,))
        H = self.h_eff(m2, terms, t)
        g = self.gamma / (1.0 + self.alpha ** 2)
        mxH = np.cross(m2, H)
        k = -g * mxH - self.alpha * g * np.cross(m2, mxH)
        return np.where(self.mass()[..., None] > 0.0, k, 0.0)

    def rk4_step(self, m2, t, dt, terms=ALL, renorm=False) -> np.ndarray:
        m = np.asarray(m2, dtype=np.float64).reshape(self.nodes + (3,))
        k1 = self.llg_rhs(m, terms, t)
        k2 = self.llg_rhs(m + 0.5 * dt * k1, terms, t + 0.5 * dt)
        k3 = self.llg_rhs(m + 0.5 * dt * k2, terms, t + 0.5 * dt)
        k4 = self.llg_rhs(m + dt * k3, terms, t + dt)
        out = m + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        if renorm:
            nrm = np.linalg.norm(out, axis=-1, keepdims=True)
            out = np.where(nrm > 0.0, out / np.where(nrm > 0.0, nrm, 1.0), out)
        return out
