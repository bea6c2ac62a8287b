"""One-dimensional nodal basis with full three-dimensional integration (section "Low-Dimensional
Geometries" of the paper) for the FP64 oracle.

TEST INFRASTRUCTURE ONLY, under the same rule as the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it.  It never imports the
CUDA library.

The 1D basis function of node i1 is the hat function of x alone, constant along y and z over all
N2 x N3 cells of the cross-section; it is the sum of the 3D nodal basis functions of the node plane
(i1, 0..N2, 0..N3), which form a partition of unity in y and z.  The 1D Galerkin system is therefore the
3D one restricted to magnetisations that depend on x alone: with m3(i1, j, k) = m1(i1),

    dE/dm1_n = sum_{j,k} dE/dm3_(n,j,k)        (chain rule)
    mass1_n  = mu0 int Ms phi1_n = sum_{j,k} mass3_(n,j,k)
    h1_n     = -dE/dm1_n / mass1_n

and the LLG right-hand side and the integrators act on the (N1+1) x 1 x 1 nodal field.  This module
evaluates exactly that, on top of the 3D oracle.
"""
from __future__ import annotations

import numpy as np

from . import ALL
from .basis2d import Mesh2D


class Mesh1D(Mesh2D):
    """N1 x N2 x N3 cells, nodal 1D basis: nodes (N1+1, 1, 1)."""

    def __init__(self, n, dx):
        super().__init__(n, dx)
        self.nodes = (self.n[0] + 1, 1, 1)

    def lift(self, m1):
        m1 = np.asarray(m1, dtype=np.float64).reshape(self.nodes + (3,))
        return np.broadcast_to(m1, (self.n[0] + 1, self.n[1] + 1, self.n[2] + 1, 3)).copy()

    def mass(self) -> np.ndarray:
        return self.m3.mass().sum(axis=(1, 2), keepdims=True)

    def variation(self, m1, terms=ALL, t=0.0) -> np.ndarray:
        return self.m3.variation(self.lift(m1), terms, t).sum(axis=(1, 2), keepdims=True)
