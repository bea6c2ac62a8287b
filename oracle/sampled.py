"""Oracle values at chosen nodes of a mesh too large for the whole-mesh oracle.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the full-size parity tests call it to get the
exact result at a sample of nodes, one by one, from the same definitions the whole-mesh oracle uses.

  - Local terms (exchange, anisotropy, Zeeman, DMI): the variation at node n involves only the cells that
    contain n, and so does its lumped mass (Eqs. weak_form_impl_f, weak_form_impl, mass_lumping).  The
    oracle's own mesh restricted to those cells therefore gives the exact field at n.
  - One explicit Runge-Kutta step with local terms only: the slope k_s at n depends on the stage input
    within one node of n, and that input on the slopes k_1..k_{s-1} there, so the 5th-order solution of
    a Dormand-Prince step (slopes 1..6) at n needs k_1 within 5 nodes, whose stencils reach the cells
    within 6.  The oracle's step on the cells within `radius` >= 6 of n gives the exact new state at n,
    provided every attempt is accepted (tolerances so loose that the error norm, which does see the cut,
    cannot reject).
  - Demagnetising field (Sec. "Demagnetization Field"): H_c = -sum_{c'} N(c - c') M_{c'} with
    M_c = Ms_c m_bar_c, summed directly over the cells where M is non-zero (a sparse source), with the
    oracle's _Float128 Newell tensor at each offset; the nodal value is the Ms-weighted mean of H_c over
    the cells holding the node (the lumped-mass form of the demag variation).  m_bar_c, the mean of the
    trilinear interpolant over the cell, is the mean of its eight corner values.
"""
from __future__ import annotations

import numpy as np

from . import Mesh, newell


def _cells_around(node, n, radius):
    """Cell box [lo, hi) of the cells within `radius` of `node`, clipped to the mesh."""
    lo = tuple(max(0, int(node[k]) - radius) for k in range(3))
    hi = tuple(min(int(n[k]), int(node[k]) + radius) for k in range(3))
    return lo, hi


def _cell_slice(v, lo, hi):
    """A scalar material value stays a scalar; a cell map is cut to the box."""
    if np.ndim(v) == 0:
        return float(v)
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64)[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]])


def submesh(n, dx, material, node, radius, zeeman=None, D=None):
    """The oracle mesh on the cells within `radius` of `node`, and the node's index in it.

    material = (Ms, A, Ku, axis, alpha, gamma) with scalars or (N1, N2, N3) cell maps; zeeman = the
    keyword arguments of ``Mesh.set_zeeman`` (cell fields as (N1, N2, N3, 3) maps); D = the DMI constant
    or cell map."""
    lo, hi = _cells_around(node, n, radius)
    Ms, A, Ku, axis, alpha, gamma = material
    me = Mesh(tuple(hi[k] - lo[k] for k in range(3)), dx)
    sub = tuple(hi[k] - lo[k] for k in range(3))
    me.set_material(np.broadcast_to(_cell_slice(Ms, lo, hi), sub).copy(),
                    np.broadcast_to(_cell_slice(A, lo, hi), sub).copy(),
                    np.broadcast_to(_cell_slice(Ku, lo, hi), sub).copy(), axis, alpha, gamma)
    if zeeman:
        z = dict(zeeman)
        if z.get("h_cell") is not None:
            z["h_cell"] = np.ascontiguousarray(np.asarray(z["h_cell"])[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]])
        me.set_zeeman(**z)
    if D is not None:
        me.set_dmi(np.broadcast_to(_cell_slice(D, lo, hi), sub).copy())
    local = tuple(int(node[k]) - lo[k] for k in range(3))
    return me, lo, hi, local


def local_field_at(n, dx, material, m, node, terms, t=0.0, zeeman=None, D=None):
    """h_eff at `node` from the local terms in `terms` (no demag), for the full nodal array m."""
    me, lo, hi, local = submesh(n, dx, material, node, 1, zeeman, D)
    m_sub = np.ascontiguousarray(m[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1], dtype=np.float64)
    return me.h_eff(m_sub, terms, t)[local]


def dp5_step_at(n, dx, material, m, node, terms, dt, radius=6):
    """The state at `node` after one accepted Dormand-Prince 5(4) step of size dt from m at t = 0, with
    local terms only, renormalised (every attempt accepted: rtol = atol = 1e3)."""
    if radius < 6:
        raise ValueError("the step at a node needs the cells within 6 nodes")
    me, lo, hi, local = submesh(n, dx, material, node, radius)
    m_sub = np.ascontiguousarray(m[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1], dtype=np.float64)
    st = me.dp5_stepper(m_sub, 0.0, dt, terms, rtol=1e3, atol=1e3, renorm=True)
    if not st.step():
        raise RuntimeError("the step was rejected")
    return st.m[local].copy()


def demag_at_nodes(n, dx, Ms, m, nodes):
    """Demag field at each node of `nodes` (a list of index triples) for a nodal m that is zero outside a
    few nodes, by direct summation over the cells where M is non-zero."""
    n = tuple(int(v) for v in n)
    Ms_of = (lambda c: float(Ms)) if np.ndim(Ms) == 0 else (lambda c: float(Ms[c]))
    # source cells: every cell with a non-zero corner, M_c = Ms_c * mean of the eight corners
    src_nodes = np.argwhere(np.any(m != 0.0, axis=-1))
    cells = set()
    for s in src_nodes:
        for i in np.ndindex(2, 2, 2):
            c = tuple(int(s[k]) - i[k] for k in range(3))
            if all(0 <= c[k] < n[k] for k in range(3)):
                cells.add(c)
    src = []
    for c in sorted(cells):
        corners = m[c[0]:c[0] + 2, c[1]:c[1] + 2, c[2]:c[2] + 2].reshape(8, 3)
        M = Ms_of(c) * corners.mean(axis=0)
        if np.any(M != 0.0):
            src.append((c, M))
    cache = {}

    def tensor(e):
        if e not in cache:
            Nv = newell(dx, (e[0] * dx[0], e[1] * dx[1], e[2] * dx[2]))
            cache[e] = np.array([[Nv[0], Nv[3], Nv[4]], [Nv[3], Nv[1], Nv[5]], [Nv[4], Nv[5], Nv[2]]])
        return cache[e]

    out = np.zeros((len(nodes), 3))
    for q, node in enumerate(nodes):
        num, den = np.zeros(3), 0.0
        for i in np.ndindex(2, 2, 2):
            c = tuple(int(node[k]) - i[k] for k in range(3))
            if not all(0 <= c[k] < n[k] for k in range(3)):
                continue
            ms = Ms_of(c)
            if ms == 0.0:
                continue
            H = np.zeros(3)
            for cs, M in src:
                H -= tensor(tuple(c[k] - cs[k] for k in range(3))) @ M
            num += ms * H
            den += ms
        out[q] = num / den if den > 0 else 0.0
    return out
