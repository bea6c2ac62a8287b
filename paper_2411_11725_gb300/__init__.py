"""GB300 (sm_103a) library for the nodal finite-difference effective field and Landau-Lifshitz-Gilbert
integration of NeuralMag (Abert et al., arXiv 2411.11725).

This package is a thin binding of the C ABI declared in ``include/nmgb.h`` (library ``libnmgb.so``
built from ``csrc/`` by ``build.py``).  Every step of the computation runs in the library's CUDA
kernels; Python only marshals arguments.  PyTorch supplies device memory and streams.

There is no CPU fallback: if the library cannot be loaded, or no CUDA device is present, the calls
raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = [
    "Mesh", "NMError", "load", "lib_path",
    "F32", "F64", "EXCH", "ANIS", "ZEE", "DEMAG", "ALL", "DMI", "RK4", "DP54",
]

OK = 0
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_STEP_UNDERFLOW, ERR_NONFINITE, ERR_TIMEOUT, ERR_STATE = -1, -2, -3, -4, -5, -6, -7
F32, F64 = 0, 1
EXCH, ANIS, ZEE, DEMAG = 1, 2, 4, 8
ALL = EXCH | ANIS | ZEE | DEMAG
DMI = 16  # interfacial DMI (nm_set_dmi); not part of ALL
RK4, DP54 = 1, 2
FIELD_HEXT_UNIFORM, FIELD_HEXT_CELL = 1, 2
MEM_HOST, MEM_DEVICE = 0, 1

_lock = threading.Lock()
_lib = None


class NMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"nm error {code}: {msg}")
        self.code = code


def lib_path() -> str:
    return _build.LIB


# (name, restype, argtypes) for every entry point of include/nmgb.h
_d, _i, _u, _l, _vp = ctypes.c_double, ctypes.c_int, ctypes.c_uint, ctypes.c_long, ctypes.c_void_p
_Pd, _Pi, _Pl = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_long)


class Request(ctypes.Structure):
    """nm_request of include/nmgb.h."""
    _fields_ = [("n", _i * 3), ("dx", _d * 3), ("precision", _i), ("Ms", _d), ("A", _d), ("Ku", _d),
                ("axis", _d * 3), ("alpha", _d), ("gamma", _d), ("h", _d * 3), ("terms", _u), ("method", _i),
                ("t_end", _d), ("rtol", _d), ("atol", _d), ("dt0", _d), ("m0", _Pd), ("m_out", _Pd),
                ("tag", _l)]


class Result(ctypes.Structure):
    """nm_result of include/nmgb.h."""
    _fields_ = [("tag", _l), ("status", _i), ("n_accepted", _l), ("n_rejected", _l), ("t_final", _d),
                ("queue_s", _d), ("run_s", _d), ("latency_s", _d), ("n_active_at_admit", _i),
                ("message", ctypes.c_char * 128)]


class ServerStats(ctypes.Structure):
    """nm_server_stats of include/nmgb.h."""
    _fields_ = [("submitted", _l), ("completed", _l), ("failed", _l), ("queued", _i), ("active", _i),
                ("pooled", _i), ("peak_active", _i), ("bytes_in_use", _l), ("peak_bytes", _l),
                ("meshes_created", _l), ("meshes_evicted", _l), ("tensor_copies", _l), ("busy_s", _d),
                ("active_s", _d), ("wall_s", _d)]

SIGNATURES = [
    ("nm_create_mesh", _i, [_i, _i, _i, _d, _d, _d, _i, _vp, ctypes.POINTER(_vp)]),
    ("nm_create_mesh_basis", _i, [_i, _i, _i, _d, _d, _d, _i, _i, _vp, ctypes.POINTER(_vp)]),
    ("nm_destroy_mesh", _i, [_vp]),
    ("nm_set_material", _i, [_vp, _Pd, _d, _Pd, _d, _Pd, _d, _Pd, _d, _d]),
    ("nm_set_field", _i, [_vp, _i, _Pd, _Pd, _d, _d]),
    ("nm_set_state", _i, [_vp, _vp, _i, _d, _d]),
    ("nm_get_state", _i, [_vp, _vp, _i, _Pd, _Pd]),
    ("nm_get_state_noalloc", _i, [_vp, _Pd, _Pd, _Pd]),
    ("nm_set_integrator", _i, [_vp, _i, _d, _i]),
    ("nm_set_error_norm", _i, [_vp, _i]),
    ("nm_measure_peak", _i, [_i, _i, _Pd]),
    ("nm_h_eff", _i, [_vp, _vp, _vp, _u, _d]),
    ("nm_set_terms", _i, [_vp, _u]),
    ("nm_set_dmi", _i, [_vp, _Pd, _d]),
    ("nm_llg_step", _i, [_vp, _i, _Pd, _Pd, _d, _d, _Pi]),
    ("nm_run_steps", _i, [_vp, _i, _l, _d, _d]),
    ("nm_get_counters", _i, [_vp, _Pl, _Pl, _Pd]),
    ("nm_mean_m", _i, [_vp, _Pd]),
    ("nm_run_until", _i, [_vp, _d, _i, _d, _d, _d, _d, _Pd, _l, _Pl, _Pl]),
    ("nm_mesh_info", _i, [_vp, _Pl, _Pl, _Pi, _Pl]),
    ("nm_profile_step", _i, [_vp, _i, _i, _d, _d, _i, _Pd, ctypes.c_char_p, _Pi]),
    ("nm_h_eff_vjp", _i, [_vp, _vp, _vp, _u, _d, _vp, _vp]),
    ("nm_adjoint_run", _i, [_vp, _i, _d, _d, _d, _d, _d, _Pd, _Pd, _i, _l, _Pd, _Pd, _Pd, _Pl, _Pd]),
    ("nm_adjoint_continuous", _i, [_vp, _d, _l, _Pd, _Pd, _Pd, _Pd, _Pd, _Pd, _Pd]),
    ("nm_footprint_bytes", _l, [_i, _i, _i, _i]),
    ("nm_sync", _i, [_vp]),
    ("nm_server_create", _i, [_l, _i, ctypes.POINTER(_vp)]),
    ("nm_server_submit", _i, [_vp, ctypes.POINTER(Request)]),
    ("nm_server_poll", _i, [_vp, ctypes.POINTER(Result), _i, _d, _Pi]),
    ("nm_server_stats_get", _i, [_vp, ctypes.POINTER(ServerStats)]),
    ("nm_server_destroy", _i, [_vp]),
    ("nm_last_error", ctypes.c_char_p, []),
]


def load(build_if_missing: bool = True):
    """Load ``libnmgb.so`` (building it first when absent) and declare every entry point."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise NMError(ERR_STATE, f"{path} not built")
            _build.build()
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc: int):
    if rc != OK:
        msg = _lib.nm_last_error().decode(errors="replace")
        raise NMError(rc, msg)


def _pd(a):
    return None if a is None else a.ctypes.data_as(_Pd)


def _host_f64(a, shape):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if a.shape != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {a.shape}")
    return a


def measure_peak(kind, reps=5) -> float:
    """FLOP/s of fused multiply-add chains on the current GPU: kind 0 FP32, 1 FP64."""
    out = np.zeros(1)
    _check(load().nm_measure_peak(int(kind), int(reps), _pd(out)))
    return float(out[0])


def footprint_bytes(n, precision=F32) -> int:
    return int(load().nm_footprint_bytes(int(n[0]), int(n[1]), int(n[2]), int(precision)))


class Mesh:
    """A mesh of N1 x N2 x N3 cuboid cells on the current CUDA device.

    Nodal fields use the layout (N1+1, N2+1, N3+1, 3); cell fields (N1, N2, N3[, 3]).  ``precision``
    is ``F32`` (FP32 field evaluation, FP64 state) or ``F64``.  ``stream`` is a ``torch.cuda.Stream``
    (default: the library creates its own stream).
    """

    def __init__(self, n, dx, precision=F32, stream=None, basis=3):
        """basis 3: trilinear nodal basis; basis 2: nodal basis constant along z over all cell layers
        (nodes (N1+1, N2+1, 1)); basis 1: nodal basis constant along y and z over the whole cross-section
        (nodes (N1+1, 1, 1)); section "Low-Dimensional Geometries"."""
        import torch
        if not torch.cuda.is_available():
            raise NMError(ERR_CUDA, "no CUDA device: this library has no CPU path")
        self._torch = torch
        self.lib = load()
        self.n = tuple(int(v) for v in n)
        self.dx = tuple(float(v) for v in dx)
        self.precision = int(precision)
        self.basis = int(basis)
        self.nodes = (self.n[0] + 1, 1 if self.basis == 1 else self.n[1] + 1, self.n[2] + 1 if self.basis == 3 else 1)
        self.dtype = torch.float64 if self.precision == F64 else torch.float32
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream
        sp = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        h = ctypes.c_void_p()
        if self.basis == 3:
            _check(self.lib.nm_create_mesh(*self.n, *self.dx, self.precision, sp, ctypes.byref(h)))
        else:
            _check(self.lib.nm_create_mesh_basis(*self.n, *self.dx, self.precision, self.basis, sp, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.nm_destroy_mesh(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------------------------------- set-up
    def info(self):
        nn, nc, by = ctypes.c_long(), ctypes.c_long(), ctypes.c_long()
        P = (ctypes.c_int * 3)()
        _check(self.lib.nm_mesh_info(self._h, ctypes.byref(nn), ctypes.byref(nc), P, ctypes.byref(by)))
        return dict(n_nodes=nn.value, n_cells=nc.value, P=tuple(P), device_bytes=by.value)

    def set_material(self, Ms, A, Ku=0.0, axis=(0.0, 0.0, 1.0), alpha=0.1, gamma=2.2127614872e5):
        def split(v):
            if np.ndim(v) == 0:
                return None, float(v)
            return _host_f64(v, self.n), 0.0
        Ms_a, Ms0 = split(Ms)
        A_a, A0 = split(A)
        Ku_a, Ku0 = split(Ku)
        ax = _host_f64(axis, (3,))
        _check(self.lib.nm_set_material(self._h, _pd(Ms_a), Ms0, _pd(A_a), A0, _pd(Ku_a), Ku0, _pd(ax),
                                        float(alpha), float(gamma)))

    def set_dmi(self, D):
        """Interfacial DMI constant (J/m^2): scalar or cell map (N1, N2, N3); enable with DMI in the terms."""
        if np.ndim(D) == 0:
            _check(self.lib.nm_set_dmi(self._h, None, float(D)))
        else:
            Dc = _host_f64(D, self.n)
            _check(self.lib.nm_set_dmi(self._h, _pd(Dc), 0.0))

    def set_zeeman(self, h_uniform=(0.0, 0.0, 0.0), freq=0.0, phase=0.0, h_cell=None, cell_freq=0.0,
                   cell_phase=0.0):
        hu = _host_f64(h_uniform, (3,))
        _check(self.lib.nm_set_field(self._h, FIELD_HEXT_UNIFORM, None, _pd(hu), float(freq), float(phase)))
        hc = None if h_cell is None else _host_f64(h_cell, self.n + (3,))
        _check(self.lib.nm_set_field(self._h, FIELD_HEXT_CELL, _pd(hc), None, float(cell_freq), float(cell_phase)))

    def set_uniform_field(self, h_uniform, freq=0.0, phase=0.0):
        """Set the uniform applied field (A/m) only, leaving any cell-wise field in place."""
        hu = _host_f64(h_uniform, (3,))
        _check(self.lib.nm_set_field(self._h, FIELD_HEXT_UNIFORM, None, _pd(hu), float(freq), float(phase)))

    def set_terms(self, terms):
        _check(self.lib.nm_set_terms(self._h, int(terms)))

    def set_integrator(self, renormalise=True, dt_min=1e-22, max_rejections=50):
        _check(self.lib.nm_set_integrator(self._h, int(bool(renormalise)), float(dt_min), int(max_rejections)))

    def set_error_norm(self, fp64_terms):
        """FP32 meshes: form the per-node terms of the Dormand-Prince error norm in FP64 (True) or FP32."""
        _check(self.lib.nm_set_error_norm(self._h, int(bool(fp64_terms))))

    # ---------------------------------------------------------------------------------- state
    def set_state(self, m, t=0.0, dt=1e-14):
        """m: numpy (host) or torch CUDA float64 tensor of shape (N1+1, N2+1, N3+1, 3)."""
        torch = self._torch
        if isinstance(m, torch.Tensor) and m.is_cuda:
            m = m.to(torch.float64).contiguous()
            if tuple(m.shape) != self.nodes + (3,):
                raise ValueError("bad shape")
            self._sync_torch()
            _check(self.lib.nm_set_state(self._h, ctypes.c_void_p(m.data_ptr()), MEM_DEVICE, float(t), float(dt)))
        else:
            a = _host_f64(m, self.nodes + (3,))
            _check(self.lib.nm_set_state(self._h, a.ctypes.data_as(ctypes.c_void_p), MEM_HOST, float(t), float(dt)))

    def get_state(self, device=False):
        """(m, t, dt); m as a numpy array, or a torch CUDA tensor when device=True."""
        t, dt = ctypes.c_double(), ctypes.c_double()
        if device:
            torch = self._torch
            out = torch.empty(self.nodes + (3,), dtype=torch.float64, device=self.device)
            self._sync_torch()
            _check(self.lib.nm_get_state(self._h, ctypes.c_void_p(out.data_ptr()), MEM_DEVICE, ctypes.byref(t),
                                         ctypes.byref(dt)))
            return out, t.value, dt.value
        out = np.empty(self.nodes + (3,))
        _check(self.lib.nm_get_state(self._h, out.ctypes.data_as(ctypes.c_void_p), MEM_HOST, ctypes.byref(t),
                                     ctypes.byref(dt)))
        return out, t.value, dt.value

    def set_state_host_ptr(self, m, t, dt):
        """Set the state from a contiguous float64 CPU torch tensor (e.g. pinned) without a copy."""
        if m.dtype != self._torch.float64 or m.is_cuda or not m.is_contiguous() or tuple(m.shape) != self.nodes + (3,):
            raise ValueError("need a contiguous float64 CPU tensor of the nodal shape")
        _check(self.lib.nm_set_state(self._h, ctypes.c_void_p(m.data_ptr()), MEM_HOST, float(t), float(dt)))

    def get_state_host_ptr(self, out):
        """Copy the state into a contiguous float64 CPU torch tensor; returns (t, dt)."""
        if out.dtype != self._torch.float64 or out.is_cuda or not out.is_contiguous() or \
                tuple(out.shape) != self.nodes + (3,):
            raise ValueError("need a contiguous float64 CPU tensor of the nodal shape")
        t, dt = ctypes.c_double(), ctypes.c_double()
        _check(self.lib.nm_get_state(self._h, ctypes.c_void_p(out.data_ptr()), MEM_HOST, ctypes.byref(t),
                                     ctypes.byref(dt)))
        return t.value, dt.value

    def mean_m(self):
        """Volume-weighted mean of the resident m (numpy array of 3)."""
        out = np.zeros(3)
        _check(self.lib.nm_mean_m(self._h, _pd(out)))
        return out

    def counters(self):
        a, r, e = ctypes.c_long(), ctypes.c_long(), ctypes.c_double()
        _check(self.lib.nm_get_counters(self._h, ctypes.byref(a), ctypes.byref(r), ctypes.byref(e)))
        return a.value, r.value, e.value

    def _sync_torch(self):
        # torch allocations and copies are ordered on torch's current stream; the library works on its own
        self._torch.cuda.current_stream().synchronize()

    def sync(self):
        _check(self.lib.nm_sync(self._h))

    # ---------------------------------------------------------------------------------- compute
    def h_eff(self, m=None, terms=ALL, t=0.0, out=None):
        """Effective field for a nodal torch CUDA tensor m (or the resident state when None)."""
        torch = self._torch
        if out is None:
            out = torch.empty(self.nodes + (3,), dtype=self.dtype, device=self.device)
        mp = None
        if m is not None:
            if not (isinstance(m, torch.Tensor) and m.is_cuda):
                raise TypeError("m must be a CUDA tensor")
            m = m.to(self.dtype).contiguous()
            if tuple(m.shape) != self.nodes + (3,):
                raise ValueError("bad shape")
            mp = ctypes.c_void_p(m.data_ptr())
        self._sync_torch()
        _check(self.lib.nm_h_eff(self._h, mp, ctypes.c_void_p(out.data_ptr()), int(terms), float(t)))
        self.sync()
        return out

    def llg_step(self, method=DP54, t=0.0, dt=1e-14, rtol=1e-5, atol=1e-5):
        tt, dd, acc = ctypes.c_double(t), ctypes.c_double(dt), ctypes.c_int(0)
        _check(self.lib.nm_llg_step(self._h, int(method), ctypes.byref(tt), ctypes.byref(dd), float(rtol),
                                    float(atol), ctypes.byref(acc)))
        return bool(acc.value), tt.value, dd.value

    def run_steps(self, n_steps, method=DP54, rtol=1e-5, atol=1e-5):
        _check(self.lib.nm_run_steps(self._h, int(method), int(n_steps), float(rtol), float(atol)))

    def profile_step(self, method=DP54, reps=3, rtol=1e-5, atol=1e-5, max_kernels=128):
        """[(kernel name, mean ms)] of one integrator step, launch by launch (CUDA events)."""
        ms = np.zeros(max_kernels)
        names = ctypes.create_string_buffer(32 * max_kernels)
        nk = ctypes.c_int()
        _check(self.lib.nm_profile_step(self._h, int(method), int(reps), float(rtol), float(atol), max_kernels,
                                        _pd(ms), names, ctypes.byref(nk)))
        raw = names.raw
        out = []
        for i in range(min(nk.value, max_kernels)):
            nm = raw[32 * i:32 * i + 32].split(b"\0")[0].decode()
            out.append((nm, float(ms[i])))
        return out

    def h_eff_vjp(self, m, v, terms=ALL, t=0.0, want_Ms=True):
        """(J_h(m)^T v, d<v, h(m)>/dMs) for nodal CUDA tensors m, v; the second is None unless want_Ms."""
        torch = self._torch
        m = m.to(self.dtype).contiguous()
        v = v.to(self.dtype).contiguous()
        gm = torch.empty(self.nodes + (3,), dtype=self.dtype, device=self.device)
        gMs = torch.empty(self.n, dtype=self.dtype, device=self.device) if want_Ms else None
        self._sync_torch()
        _check(self.lib.nm_h_eff_vjp(self._h, ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                     int(terms), float(t), ctypes.c_void_p(gm.data_ptr()),
                                     None if gMs is None else ctypes.c_void_p(gMs.data_ptr())))
        self.sync()
        return gm, gMs

    def adjoint_run(self, t_end, weight, target=None, method=DP54, rtol=1e-5, atol=1e-5, dt0=0.0,
                    sample_dt=0.0, include_initial=False, checkpoint_every=32, field_grad=False, loss_only=False):
        """Forward integration to t_end with the sampled quadratic loss and its discrete adjoint.
        Returns (loss, dL/dMs (N1,N2,N3), dL/dm0 nodal, accepted steps), and dL/dh of the uniform applied
        field (3,) as a fifth element when field_grad is set.  loss_only: the forward run alone; the
        gradients come back as None."""
        W = _host_f64(weight, self.nodes + (3,))
        tg = None if target is None else _host_f64(target, self.nodes + (3,))
        loss = ctypes.c_double()
        gMs = None if loss_only else np.zeros(self.n)
        gm0 = None if loss_only else np.zeros(self.nodes + (3,))
        gh = np.zeros(3) if (field_grad and not loss_only) else None
        ns = ctypes.c_long()
        _check(self.lib.nm_adjoint_run(self._h, int(method), float(t_end), float(rtol), float(atol), float(dt0),
                                       float(sample_dt), _pd(W), _pd(tg), int(bool(include_initial)),
                                       int(checkpoint_every), ctypes.byref(loss), _pd(gMs), _pd(gm0),
                                       ctypes.byref(ns), _pd(gh)))
        if field_grad:
            return loss.value, gMs, gm0, ns.value, gh
        return loss.value, gMs, gm0, ns.value

    def adjoint_continuous(self, t_end, n_steps, weight, target=None):
        """Forward RK4 (n_steps) to t_end with the final-time quadratic loss, then the continuous adjoint
        system integrated backwards.  Returns (loss, dL/dm0 nodal, dL/dMs (N1,N2,N3), dL/dh (3,),
        reconstructed m(t0) nodal)."""
        W = _host_f64(weight, self.nodes + (3,))
        tg = None if target is None else _host_f64(target, self.nodes + (3,))
        loss = ctypes.c_double()
        gm0 = np.zeros(self.nodes + (3,))
        gMs = np.zeros(self.n)
        gh = np.zeros(3)
        m0r = np.zeros(self.nodes + (3,))
        _check(self.lib.nm_adjoint_continuous(self._h, float(t_end), int(n_steps), _pd(W), _pd(tg),
                                              ctypes.byref(loss), _pd(gm0), _pd(gMs), _pd(gh), _pd(m0r)))
        return loss.value, gm0, gMs, gh, m0r

    def run_until(self, t_end, method=DP54, rtol=1e-5, atol=1e-5, dt0=0.0, sample_dt=0.0):
        """Integrate to t_end; returns (samples (k,3) or None, n_accepted, n_rejected)."""
        t = self.get_state()[1]
        samples = None
        ns = 0
        if sample_dt > 0:
            ns = int(np.floor((t_end - t) / sample_dt * (1 + 1e-12))) + 1
            samples = np.zeros((ns, 3))
        na, nr = ctypes.c_long(), ctypes.c_long()
        _check(self.lib.nm_run_until(self._h, float(t_end), int(method), float(rtol), float(atol), float(dt0),
                                     float(sample_dt), _pd(samples), ns, ctypes.byref(na), ctypes.byref(nr)))
        return samples, na.value, nr.value
