"""FP64 CPU oracle for the nodal finite-difference effective field and LLG integration
(NeuralMag, arXiv 2411.11725).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
(``paper_2411_11725_gb300``) and never imports it; the C source ``nm_oracle.c`` is compiled here with
gcc and called through ctypes.

Layouts follow the paper's tensors (C order, FP64): nodal vector fields ``(N1+1, N2+1, N3+1, 3)``,
cell scalars ``(N1, N2, N3)``, cell vectors ``(N1, N2, N3, 3)``.

Parity unpinned: the value of gamma and the physical choices of each workload are conventions passed
in by the caller.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MU0 = 4e-7 * np.pi
EXCH, ANIS, ZEE, DEMAG = 1, 2, 4, 8
ALL = EXCH | ANIS | ZEE | DEMAG
DMI = 16  # interfacial DMI (a reading: the paper names antisymmetric exchange without its energy)


def build(force: bool = False) -> str:
    """Compile ``nm_oracle.c`` into ``liboracle.so`` next to it (gcc, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off", "-std=gnu11",
               "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d, i, u, vp = ctypes.c_double, ctypes.c_int, ctypes.c_uint, ctypes.c_void_p
        P = ctypes.POINTER(ctypes.c_double)
        lib.or_create.restype = vp
        lib.or_create.argtypes = [i, i, i, d, d, d]
        lib.or_free.argtypes = [vp]
        lib.or_set_material.argtypes = [vp, P, P, P, P, d, d]
        lib.or_set_zeeman.argtypes = [vp, P, d, d, P, d, d]
        lib.or_set_dmi.argtypes = [vp, P]
        lib.or_mass.argtypes = [vp, P]
        lib.or_newell.argtypes = [d, d, d, d, d, d, P]
        lib.or_compute_tensor.argtypes = [vp]
        lib.or_get_tensor.argtypes = [vp, P]
        lib.or_demag_cells.argtypes = [vp, P, P]
        lib.or_variation.argtypes = [vp, P, u, d, P]
        lib.or_h_eff.argtypes = [vp, P, u, d, P]
        lib.or_energy.argtypes = [vp, P, u, d]
        lib.or_energy.restype = d
        lib.or_llg_rhs.argtypes = [vp, P, u, d, P]
        lib.or_rk4_step.argtypes = [vp, P, u, d, d, i]
        lib.or_dp5_step.argtypes = [vp, P, P, ctypes.POINTER(i), u, P, P, d, d, i, P]
        lib.or_dp5_step.restype = i
        lib.or_dp5_tableau.argtypes = [P, P, P, P]
        lib.or_element_matrices.argtypes = [d, d, d, P, P, P]
        lib.or_phi.argtypes = [i, d, d, d]
        lib.or_phi.restype = d
        lib.or_num_threads.restype = i
        lib.or_set_num_threads.argtypes = [i]
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None and a.shape != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {a.shape}")
    return a


def num_threads() -> int:
    return _load().or_num_threads()


def set_num_threads(n: int) -> None:
    """Thread count for the oracle's parallel loops (its results do not depend on it)."""
    _load().or_set_num_threads(int(n))


def phi(li: int, x1: float, x2: float, x3: float) -> float:
    """Reference trilinear basis function of local vertex li = 4 i1 + 2 i2 + i3 (Eq. nodal_basis)."""
    return _load().or_phi(li, x1, x2, x3)


def element_matrices(dx):
    """(Kex, Mm, Phi): int 2 grad(phi_i).grad(phi_j), int phi_i phi_j, int phi_i over one cell (8x8, 8x8, 8)."""
    K = np.zeros(64); M = np.zeros(64); Phi = np.zeros(8)
    _load().or_element_matrices(float(dx[0]), float(dx[1]), float(dx[2]), _p(K), _p(M), _p(Phi))
    return K.reshape(8, 8), M.reshape(8, 8), Phi


def newell(dx, offset) -> np.ndarray:
    """Newell tensor (Nxx, Nyy, Nzz, Nxy, Nxz, Nyz) of two dx-cuboids at physical offset (X, Y, Z)."""
    out = np.zeros(6)
    _load().or_newell(float(dx[0]), float(dx[1]), float(dx[2]),
                      float(offset[0]), float(offset[1]), float(offset[2]), _p(out))
    return out


def dp5_tableau():
    c = np.zeros(7); a = np.zeros(42); b = np.zeros(7); bs = np.zeros(7)
    _load().or_dp5_tableau(_p(c), _p(a), _p(b), _p(bs))
    return c, a.reshape(7, 6), b, bs


class Mesh:
    """A cuboid mesh of N1 x N2 x N3 cells of size dx (Sec. "Nodal Finite-Difference Scheme")."""

    def __init__(self, n, dx):
        self.n = tuple(int(v) for v in n)
        self.dx = tuple(float(v) for v in dx)
        self._lib = _load()
        self._h = self._lib.or_create(*self.n, *self.dx)
        if not self._h:
            raise ValueError("invalid mesh")
        self.cells = self.n
        self.nodes = tuple(v + 1 for v in self.n)
        self._keep = []

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_free(h)
            self._h = None

    # -- setup --------------------------------------------------------------------------------
    def set_material(self, Ms, A, Ku=0.0, axis=(0.0, 0.0, 1.0), alpha=0.0, gamma=0.0):
        cs = self.cells
        Ms = _f64(np.broadcast_to(np.asarray(Ms, dtype=np.float64), cs))
        A = _f64(np.broadcast_to(np.asarray(A, dtype=np.float64), cs))
        Ku = _f64(np.broadcast_to(np.asarray(Ku, dtype=np.float64), cs))
        ax = _f64(axis, (3,))
        self._lib.or_set_material(self._h, _p(Ms), _p(A), _p(Ku), _p(ax), float(alpha), float(gamma))
        self.alpha, self.gamma = float(alpha), float(gamma)

    def set_zeeman(self, h_uniform=(0.0, 0.0, 0.0), freq=0.0, phase=0.0, h_cell=None, cell_freq=0.0,
                   cell_phase=0.0):
        hu = _f64(h_uniform, (3,))
        hc = None if h_cell is None else _f64(h_cell, self.cells + (3,))
        self._lib.or_set_zeeman(self._h, _p(hu), float(freq), float(phase),
                                None if hc is None else _p(hc), float(cell_freq), float(cell_phase))

    def set_dmi(self, D):
        """Interfacial DMI constant D (J/m^2), scalar or per cell: E = int D [m_z div m - (m.grad) m_z]."""
        Dc = _f64(np.broadcast_to(np.asarray(D, dtype=np.float64), self.cells))
        self._lib.or_set_dmi(self._h, _p(Dc))

    # -- fields -------------------------------------------------------------------------------
    def _m(self, m):
        return _f64(m, self.nodes + (3,))

    def mass(self) -> np.ndarray:
        out = np.zeros(self.nodes)
        self._lib.or_mass(self._h, _p(out))
        return out

    def tensor(self) -> np.ndarray:
        """Demag tensor octant for offsets [0,N1) x [0,N2) x [0,N3): shape (N1, N2, N3, 6)."""
        out = np.zeros(self.cells + (6,))
        self._lib.or_get_tensor(self._h, _p(out))
        return out

    def demag_cells(self, m) -> np.ndarray:
        m = self._m(m)
        out = np.zeros(self.cells + (3,))
        self._lib.or_demag_cells(self._h, _p(m), _p(out))
        return out

    def variation(self, m, terms=ALL, t=0.0) -> np.ndarray:
        m = self._m(m)
        out = np.zeros(self.nodes + (3,))
        self._lib.or_variation(self._h, _p(m), terms, float(t), _p(out))
        return out

    def h_eff(self, m, terms=ALL, t=0.0) -> np.ndarray:
        m = self._m(m)
        out = np.zeros(self.nodes + (3,))
        self._lib.or_h_eff(self._h, _p(m), terms, float(t), _p(out))
        return out

    def energy(self, m, terms=ALL, t=0.0) -> float:
        m = self._m(m)
        return self._lib.or_energy(self._h, _p(m), terms, float(t))

    def llg_rhs(self, m, terms=ALL, t=0.0) -> np.ndarray:
        m = self._m(m)
        out = np.zeros(self.nodes + (3,))
        self._lib.or_llg_rhs(self._h, _p(m), terms, float(t), _p(out))
        return out

    # -- integrators ---------------------------------------------------------------------------
    def rk4_step(self, m, t, dt, terms=ALL, renorm=False) -> np.ndarray:
        m = self._m(m).copy()
        self._lib.or_rk4_step(self._h, _p(m), terms, float(t), float(dt), int(bool(renorm)))
        return m

    def dp5_stepper(self, m, t, dt, terms=ALL, rtol=1e-5, atol=1e-5, renorm=True):
        return _DP5(self, m, t, dt, terms, rtol, atol, renorm)


class _DP5:
    """Adaptive Dormand-Prince stepping with FSAL (see or_dp5_step in nm_oracle.c)."""

    def __init__(self, mesh, m, t, dt, terms, rtol, atol, renorm):
        self.mesh = mesh
        self.m = mesh._m(m).copy()
        self.k1 = np.zeros_like(self.m)
        self.k1_valid = ctypes.c_int(0)
        self.t = ctypes.c_double(t)
        self.dt = ctypes.c_double(dt)
        self.terms, self.rtol, self.atol, self.renorm = terms, rtol, atol, renorm
        self.n_acc = 0
        self.n_rej = 0
        self.err = 0.0

    def step(self) -> bool:
        err = ctypes.c_double(0.0)
        acc = self.mesh._lib.or_dp5_step(self.mesh._h, _p(self.m), _p(self.k1), ctypes.byref(self.k1_valid),
                                         self.terms, ctypes.byref(self.t), ctypes.byref(self.dt),
                                         float(self.rtol), float(self.atol), int(bool(self.renorm)),
                                         ctypes.byref(err))
        self.err = err.value
        if acc:
            self.n_acc += 1
        else:
            self.n_rej += 1
        return bool(acc)

    def set_dt(self, dt):
        self.dt.value = float(dt)
