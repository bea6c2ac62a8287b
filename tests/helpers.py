"""Shared test helpers: set up the same Problem on the oracle and on the GPU library."""
import math

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


def aharoni_Dz(a, b, c):
    """Demagnetising factor along c of a prism with half-sides a, b, c (Aharoni 1998)."""
    abc = math.sqrt(a * a + b * b + c * c)
    ab = math.sqrt(a * a + b * b)
    bc = math.sqrt(b * b + c * c)
    ac = math.sqrt(a * a + c * c)
    t = ((b * b - c * c) / (2 * b * c) * math.log((abc - a) / (abc + a))
         + (a * a - c * c) / (2 * a * c) * math.log((abc - b) / (abc + b))
         + b / (2 * c) * math.log((ab + a) / (ab - a))
         + a / (2 * c) * math.log((ab + b) / (ab - b))
         + c / (2 * a) * math.log((bc - b) / (bc + b))
         + c / (2 * b) * math.log((ac - a) / (ac + a))
         + 2 * math.atan(a * b / (c * abc))
         + (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
         + (a * a + b * b - 2 * c * c) / (3 * a * b * c) * abc
         + c / (a * b) * (ac + bc)
         - (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c))
    return t / math.pi


def aharoni_factors(L):
    """Demagnetising factors (Dx, Dy, Dz) of a prism with side lengths L."""
    hx, hy, hz = L[0] / 2, L[1] / 2, L[2] / 2
    return np.array([aharoni_Dz(hy, hz, hx), aharoni_Dz(hz, hx, hy), aharoni_Dz(hx, hy, hz)])
