"""Shared test helpers: set up the same Problem on the oracle and on the GPU library."""
import numpy as np

import nm_inputs as inp


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.linalg.norm((a - b).ravel())
    n = np.linalg.norm(b.ravel())
    return d / n if n > 0 else d


def oracle_mesh(oracle, p: inp.Problem):
    me = oracle.Mesh(p.n, p.dx)
    me.set_material(p.Ms_cells(), p.A_cells(), p.Ku_cells(), p.axis, p.alpha, p.gamma)
    me.set_zeeman(p.h_uniform, p.h_freq, p.h_phase, p.h_cell, p.cell_freq, p.cell_phase)
    return me


def gpu_mesh(nmgb, p: inp.Problem, precision):
    me = nmgb.Mesh(p.n, p.dx, precision)
    def arg(v):
        return v if np.ndim(v) == 0 else np.asarray(v, dtype=np.float64)
    me.set_material(arg(p.Ms), arg(p.A), arg(p.Ku), p.axis, p.alpha, p.gamma)
    me.set_zeeman(p.h_uniform, p.h_freq, p.h_phase, p.h_cell, p.cell_freq, p.cell_phase)
    me.set_terms(p.terms)
    return me


def rounded(m, precision):
    """The input the GPU sees, promoted back to FP64 for the oracle (isolates kernel error)."""
    return np.asarray(m, dtype=np.float32).astype(np.float64) if precision == 0 else np.asarray(m, np.float64)
