"""Serving: many independent LLG runs of different grid sizes and materials on one GPU.

``Server`` binds the request loop of the C ABI (``nm_server_*`` in ``include/nmgb.h``): a worker thread
in the library admits queued requests as run slots and HBM budget free up, keeps each admitted run's
magnetisation and RK state resident on the device, and steps the runs on separate CUDA streams so that
their kernels overlap.  Each run is the library's single-mesh integration (the LLG equation with the
adaptive Dormand-Prince or the RK4 integrator), so a result does not depend on the other runs.

``replay`` submits a list of requests at their arrival times (seconds after the start) and collects the
results, for load tests with Poisson arrivals.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import (DEMAG, DP54, EXCH, F32, ZEE, NMError, Request, Result, ServerStats, _check, _host_f64,
               ERR_CUDA, load)

GAMMA = 4e-7 * np.pi * 1.76085963023e11


class Server:
    """Request loop on the current CUDA device.

    hbm_budget_bytes: upper bound on the summed footprints of the meshes the server holds (running or
    idle, see ``footprint_bytes``); max_active: runs on the device at once.
    """

    def __init__(self, hbm_budget_bytes: int, max_active: int = 16):
        import torch
        if not torch.cuda.is_available():
            raise NMError(ERR_CUDA, "no CUDA device: this library has no CPU path")
        self._torch = torch
        self.lib = load()
        h = ctypes.c_void_p()
        _check(self.lib.nm_server_create(int(hbm_budget_bytes), int(max_active), ctypes.byref(h)))
        self._h = h
        self._pending = {}
        self._next_tag = 0

    def submit(self, n, dx, m0, t_end, Ms, A, Ku=0.0, axis=(0.0, 0.0, 1.0), alpha=0.1, gamma=GAMMA,
               h=(0.0, 0.0, 0.0), terms=EXCH | ZEE | DEMAG, method=DP54, rtol=1e-5, atol=1e-5, dt0=1e-14,
               precision=F32, tag=None, want_m=True) -> int:
        """Queue one run from t = 0 to t_end; returns its tag.  m0: host (N1+1, N2+1, N3+1, 3)."""
        n = tuple(int(v) for v in n)
        nodes = tuple(v + 1 for v in n)
        m0 = _host_f64(m0, nodes + (3,))
        m_out = self._torch.empty(nodes + (3,), dtype=self._torch.float64, pin_memory=True) if want_m else None
        if tag is None:
            tag = self._next_tag
        self._next_tag = max(self._next_tag, int(tag)) + 1
        if int(tag) in self._pending:
            raise ValueError(f"tag {tag} is still pending")
        r = Request()
        r.n = (ctypes.c_int * 3)(*n)
        r.dx = (ctypes.c_double * 3)(*[float(v) for v in dx])
        r.precision = int(precision)
        r.Ms, r.A, r.Ku = float(Ms), float(A), float(Ku)
        r.axis = (ctypes.c_double * 3)(*[float(v) for v in axis])
        r.alpha, r.gamma = float(alpha), float(gamma)
        r.h = (ctypes.c_double * 3)(*[float(v) for v in h])
        r.terms = int(terms)
        r.method = int(method)
        r.t_end, r.rtol, r.atol, r.dt0 = float(t_end), float(rtol), float(atol), float(dt0)
        r.m0 = m0.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        r.m_out = None if m_out is None else ctypes.cast(ctypes.c_void_p(m_out.data_ptr()),
                                                         ctypes.POINTER(ctypes.c_double))
        r.tag = int(tag)
        # the library borrows m0 and m_out until the result is returned: keep them alive until then
        self._pending[int(tag)] = (m0, m_out)
        rc = self.lib.nm_server_submit(self._h, ctypes.byref(r))
        if rc != 0:
            del self._pending[int(tag)]
            _check(rc)
        return int(tag)

    def poll(self, wait_s: float = 0.0, max_results: int = 64) -> list:
        """Finished results (dicts with tag, status, counters, timings and ``m`` = m(t_end) as numpy)."""
        buf = (Result * max_results)()
        n = ctypes.c_int()
        _check(self.lib.nm_server_poll(self._h, buf, int(max_results), float(wait_s), ctypes.byref(n)))
        out = []
        for i in range(n.value):
            r = buf[i]
            m0, m_out = self._pending.pop(int(r.tag), (None, None))
            out.append(dict(tag=int(r.tag), status=int(r.status), n_accepted=int(r.n_accepted),
                            n_rejected=int(r.n_rejected), t_final=float(r.t_final), queue_s=float(r.queue_s),
                            run_s=float(r.run_s), latency_s=float(r.latency_s),
                            n_active_at_admit=int(r.n_active_at_admit),
                            message=r.message.decode(errors="replace"),
                            m=None if m_out is None else m_out.numpy()))
        return out

    def stats(self) -> dict:
        s = ServerStats()
        _check(self.lib.nm_server_stats_get(self._h, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in ServerStats._fields_}

    def drain(self, count: int, timeout_s: float = 600.0) -> list:
        """Collect ``count`` results (raises TimeoutError when they do not arrive in time)."""
        out = []
        t_stop = time.perf_counter() + timeout_s
        while len(out) < count:
            left = t_stop - time.perf_counter()
            if left <= 0:
                raise TimeoutError(f"{len(out)} of {count} results after {timeout_s} s")
            out += self.poll(wait_s=min(left, 0.5))
        return out

    @property
    def pending(self) -> int:
        return len(self._pending)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.nm_server_destroy(self._h)
            self._h = None
            self._pending.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def replay(server: Server, stream, time_scale: float = 1.0, timeout_s: float = 600.0) -> list:
    """Submit ``stream`` = [(arrival_s, submit_kwargs), ...] at arrival_s * time_scale seconds after the
    start (in real time) and return every result, in completion order."""
    order = sorted(range(len(stream)), key=lambda i: stream[i][0])
    results = []
    t0 = time.perf_counter()
    t_stop = t0 + timeout_s
    k = 0
    while k < len(order) or server.pending:
        now = time.perf_counter()
        if now > t_stop:
            raise TimeoutError(f"{len(results)} of {len(stream)} results after {timeout_s} s")
        while k < len(order) and stream[order[k]][0] * time_scale <= now - t0:
            server.submit(**stream[order[k]][1])
            k += 1
        if k < len(order):
            wait = max(0.0, stream[order[k]][0] * time_scale - (time.perf_counter() - t0))
            results += server.poll(wait_s=min(wait, 0.05))
        else:
            results += server.poll(wait_s=0.05)
    return results
