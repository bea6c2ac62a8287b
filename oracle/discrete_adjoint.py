"""Reference gradients of the discrete forward map for the FP64 oracle: backpropagation through the
integrator with the step sizes of the forward run frozen (section "Automatic Differentiation and Time
Integration"), for the cell Ms map (Eq. ms_discrete) and the initial magnetisation, the design
variables of the inverse problem (Eq. inverse_min).

TEST INFRASTRUCTURE ONLY, under the same rule as the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it.  It never imports the
CUDA library.

The loss is the sampled quadratic loss
    L = sum_k sum_{n,j} W_{n,j} (m_{n,j}(t_k) - target_{n,j})^2
over sample times t_k = t0 + k sample_dt (k >= 1, and k = 0 when include_initial), or over t_end
alone when sample_dt <= 0.  The steps are those of an adaptive Dormand-Prince run (or fixed RK4 steps)
clipped to the sample times; once the plan is made, the step sizes are frozen and every step is
accepted, which makes L a smooth function of (Ms, m0).

Two routes to the gradient, sharing nothing but the oracle's right-hand side:
  * fd_gradient: brute-force central differences (fourth-order, four points) of the oracle's own C
    forward steps (or_rk4_step, or_dp5_step) component by component;
  * reverse_gradient: reverse mode through the stages of every step with dense Jacobians: the LLG
    Jacobian of ``oracle.adjoint`` (product rule per node on the linear field Jacobian) and the Ms
    derivative of the field built from the oracle's lumped mass, its field and the demag operator,
    which is assembled column by column from the oracle's direct demag sum.
Both are feasible on small grids only (dense Jacobians of 3 x nodes rows).

Dormand-Prince with FSAL: the first slope of a step is the last slope of the previous one, taken at
the fifth-order solution before renormalisation; the first step's first slope is f(t0, m0).  The
renormalisation m <- v/|v| follows every accepted step when renorm is set.
"""
from __future__ import annotations

import numpy as np

from . import DEMAG, MU0, ZEE, Mesh, dp5_tableau
from .adjoint import ContinuousAdjoint

RK4, DP54 = 0, 1
_RK4_C = (0.0, 0.5, 0.5, 1.0)
_RK4_A = ((), (0.5,), (0.0, 0.5), (0.0, 0.0, 1.0))
_RK4_B = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)


# ------------------------------------------------------------------------------------------------
# step plan
# ------------------------------------------------------------------------------------------------
def step_plan(mesh, m0, t0, t_end, method, dt0, rtol=1e-5, atol=1e-5, sample_dt=0.0, terms=15, renorm=True):
    """Accepted steps of the forward run: a list of (t_start, dt, ends_at_sample).

    The run goes from t0 towards the next sample time (or t_end); each attempted step is clipped to
    it.  RK4 takes steps of dt0 (clipped); Dormand-Prince starts from dt0 and continues with the
    controller's proposal (accept when err <= 1, dt <- dt clamp(0.9 err^-1/5, 0.2, 5)).  A sample
    time is reached when t is within 1e-12 |t_end| of it."""
    m = np.array(m0, dtype=np.float64).reshape(mesh.nodes + (3,))
    tiny = 1e-12 * abs(t_end)
    plan = []
    t, dt, ks = float(t0), float(dt0), 1
    st = mesh.dp5_stepper(m, t0, dt0, terms, rtol, atol, renorm) if method == DP54 else None
    while t < t_end - tiny:
        target = t_end
        if sample_dt > 0:
            target = min(target, t0 + ks * sample_dt)
        while True:
            h = min(dt0 if method == RK4 else dt, target - t)
            if method == RK4:
                m = mesh.rk4_step(m, t, h, terms, renorm)
                plan.append([t, h, False])
                t = t + h
            else:
                st.t.value, st.dt.value = t, h
                if st.step():
                    plan.append([t, h, False])
                    t = st.t.value
                dt = st.dt.value
            if t >= target - tiny:
                break
        if sample_dt <= 0:
            is_sample = t >= t_end - tiny
        else:
            is_sample = abs(t - (t0 + ks * sample_dt)) <= tiny + 1e-9 * sample_dt
        if is_sample:
            if plan:
                plan[-1][2] = True
            ks += 1
    return [tuple(s) for s in plan]


def _sample_loss(m, W, tgt):
    d = m - tgt
    return float(np.sum(W * d * d)), 2.0 * W * d


# ------------------------------------------------------------------------------------------------
# brute force: central differences of the oracle's forward steps
# ------------------------------------------------------------------------------------------------
def frozen_loss(mesh, m0, plan, W, target=None, include_initial=False, method=DP54, terms=15, renorm=True):
    """L of the run that takes exactly the planned steps with the oracle's C steppers (every step
    accepted: Dormand-Prince with tolerances so loose that the error test always passes)."""
    W = np.asarray(W, dtype=np.float64).reshape(mesh.nodes + (3,))
    tgt = np.zeros_like(W) if target is None else np.asarray(target, dtype=np.float64).reshape(W.shape)
    m = np.array(m0, dtype=np.float64).reshape(W.shape)
    loss = _sample_loss(m, W, tgt)[0] if include_initial else 0.0
    st = mesh.dp5_stepper(m, plan[0][0] if plan else 0.0, 1.0, terms, 1e300, 1e300, renorm) if method == DP54 else None
    for t, dt, is_sample in plan:
        if method == RK4:
            m = mesh.rk4_step(m, t, dt, terms, renorm)
        else:
            st.t.value, st.dt.value = t, dt
            if not st.step():
                raise RuntimeError("frozen Dormand-Prince step rejected")
            m = st.m
        if is_sample:
            loss += _sample_loss(m, W, tgt)[0]
    return loss


def fd_gradient(make_mesh, Ms, m0, plan, W, target=None, include_initial=False, method=DP54, terms=15,
                renorm=True, ms_cells=None, m0_components=None, rel_step_Ms=1e-3, step_m0=1e-4):
    """Fourth-order central differences of frozen_loss:
        g ~ (L(-2e) - 8 L(-e) + 8 L(e) - L(2e)) / (12 e)
    make_mesh(Ms) returns an oracle mesh with that cell Ms map, everything else fixed (it may hand back
    the same mesh object each time, re-materialised).  ms_cells /
    m0_components restrict the components (index tuples); None = all.  Components not evaluated are
    NaN.  The Ms step is rel_step_Ms * Ms_c, the m0 step is step_m0."""
    Ms = np.asarray(Ms, dtype=np.float64)
    m0 = np.asarray(m0, dtype=np.float64)

    def L(mesh, m):
        return frozen_loss(mesh, m, plan, W, target, include_initial, method, terms, renorm)

    gMs = np.full(Ms.shape, np.nan)
    cells = list(np.ndindex(*Ms.shape)) if ms_cells is None else [tuple(c) for c in ms_cells]
    for c in cells:
        e = rel_step_Ms * Ms[c]
        vals = []
        for k in (-2, -1, 1, 2):
            M2 = Ms.copy()
            M2[c] += k * e
            vals.append(L(make_mesh(M2), m0))
        gMs[c] = (vals[0] - 8.0 * vals[1] + 8.0 * vals[2] - vals[3]) / (12.0 * e)
    gm0 = np.full(m0.shape, np.nan)
    base = make_mesh(Ms)
    comps = list(np.ndindex(*m0.shape)) if m0_components is None else [tuple(c) for c in m0_components]
    for c in comps:
        vals = []
        for k in (-2, -1, 1, 2):
            m2 = m0.copy()
            m2[c] += k * step_m0
            vals.append(L(base, m2))
        gm0[c] = (vals[0] - 8.0 * vals[1] + 8.0 * vals[2] - vals[3]) / (12.0 * step_m0)
    return gMs, gm0


# ------------------------------------------------------------------------------------------------
# reverse mode with dense Jacobians
# ------------------------------------------------------------------------------------------------
def _time_factor(freq, phase, t):
    """s(t) of the applied field: 1 for a static field, sin(2 pi f t + phase) otherwise."""
    return 1.0 if freq == 0.0 else np.sin(2.0 * np.pi * freq * t + phase)


def demag_operator(n, dx):
    """G with H_c = sum_c' G[c, :, c', :] M_c' for the cell moments M_c' = Ms_c' mbar_c' (shape
    (Nc, 3, Nc, 3), cells in C order).  Column (c', j) is the oracle's direct demag sum on a mesh
    whose only magnetic cell is c' (Ms = 1) for a uniform nodal field e_j (so mbar_c' = e_j)."""
    nc = int(np.prod(n))
    G = np.zeros((nc, 3, nc, 3))
    nodes = tuple(v + 1 for v in n)
    me = Mesh(n, dx)
    for c in range(nc):
        Ms = np.zeros(nc)
        Ms[c] = 1.0
        me.set_material(Ms.reshape(n), 0.0, 0.0)
        for j in range(3):
            m = np.zeros(nodes + (3,))
            m[..., j] = 1.0
            G[:, :, c, j] = me.demag_cells(m).reshape(nc, 3)
    return G


def cell_mean(m):
    """Mean of the 8 corners of every cell (= the cell mean of the trilinear interpolant): (N1,N2,N3,3)."""
    return 0.125 * sum(m[i1:m.shape[0] - 1 + i1, i2:m.shape[1] - 1 + i2, i3:m.shape[2] - 1 + i3]
                       for i1 in (0, 1) for i2 in (0, 1) for i3 in (0, 1))


def corner_sum(r):
    """Sum over the 8 corner nodes of every cell of a nodal field: (N1+1,N2+1,N3+1,...) -> (N1,N2,N3,...)."""
    return sum(r[i1:r.shape[0] - 1 + i1, i2:r.shape[1] - 1 + i2, i3:r.shape[2] - 1 + i3]
               for i1 in (0, 1) for i2 in (0, 1) for i3 in (0, 1))


class DiscreteAdjoint:
    """Reverse-mode gradient of the sampled loss of one oracle mesh, material and term set.

    ``zeeman`` = (h_uniform, freq, phase, h_cell or None, cell_freq, cell_phase) as given to
    ``Mesh.set_zeeman`` (needed for the cell-wise source of the Ms derivative).  The mesh must have no
    vacuum cells (Ms > 0 everywhere: the field is not differentiable in Ms where a cell switches on)."""

    def __init__(self, mesh, Ms, zeeman, terms=15):
        self.mesh = mesh
        self.terms = terms
        self.n = mesh.n
        self.nodes = mesh.nodes
        self.Ms = np.asarray(Ms, dtype=np.float64).reshape(self.n)
        if not np.all(self.Ms > 0):
            raise ValueError("reverse_gradient needs Ms > 0 in every cell")
        self.ca = ContinuousAdjoint(mesh, terms)
        self.mass = mesh.mass()
        self.w8 = MU0 * float(np.prod(mesh.dx)) / 8.0  # mu0 times the integral of one corner's basis function
        self.G = demag_operator(self.n, mesh.dx) if terms & DEMAG else None
        self.zeeman = zeeman

    # f and its transpose products ---------------------------------------------------------------
    def f(self, y, t):
        return self.mesh.llg_rhs(y, self.terms, t)

    def _cell_source(self, t):
        """Applied field per cell (uniform part plus cell part) at time t, (N1,N2,N3,3)."""
        hu, fu, pu, hc, fc, pc = self.zeeman
        S = np.broadcast_to(np.asarray(hu, dtype=np.float64) * _time_factor(fu, pu, t), self.n + (3,)).copy()
        if hc is not None:
            S += np.asarray(hc, dtype=np.float64).reshape(self.n + (3,)) * _time_factor(fc, pc, t)
        return S

    def vjp(self, y, t, v):
        """((df/dm)^T v, (df/dMs)^T v) at (y, t) for a nodal v."""
        y = y.reshape(self.nodes + (3,))
        Dm, DH = self.ca.blocks(y.reshape(-1), t)
        vv = v.reshape(-1, 3)
        q = np.einsum("nji,nj->ni", DH, vv)  # (df_n/dH_n)^T v_n
        gm = np.einsum("nji,nj->ni", Dm, vv).reshape(-1) + self.ca.Jh.T @ q.reshape(-1)
        # H_n = (-dE_loc,n + w8 sum_{c∋n} Ms_c S_c) / mass_n with S_c the cell source (applied + demag)
        H = self.ca.field(y.reshape(-1), t).reshape(self.nodes + (3,))
        r = np.zeros(self.nodes + (3,))
        mag = self.mass > 0
        r[mag] = q.reshape(self.nodes + (3,))[mag] / self.mass[mag][:, None]
        S = np.zeros(self.n + (3,))
        if self.terms & ZEE:
            S += self._cell_source(t)
        if self.terms & DEMAG:
            S += self.mesh.demag_cells(y)
        # direct part: d H_n / d Ms_c = w8 (S_c - H_n) / mass_n for the corners n of c
        g = self.w8 * (np.einsum("abcj,abcj->abc", corner_sum(r), S) - corner_sum(np.sum(r * H, axis=-1)))
        if self.terms & DEMAG:
            # through the demag source M_c = Ms_c mbar_c: sum_{c'} (Ms_c' R_c') . G[c', c] mbar_c
            nc = int(np.prod(self.n))
            R = corner_sum(r).reshape(nc, 3) * self.Ms.reshape(nc, 1)
            GR = np.einsum("aibj,ai->bj", self.G, R)
            g = g + self.w8 * np.einsum("bj,bj->b", GR, cell_mean(y).reshape(nc, 3)).reshape(self.n)
        return gm.reshape(self.nodes + (3,)), g

    # reverse sweep ------------------------------------------------------------------------------
    def reverse_gradient(self, m0, plan, W, target=None, include_initial=False, method=DP54, renorm=True):
        """(loss, dL/dMs (N1,N2,N3), dL/dm0 nodal) of the planned run."""
        W = np.asarray(W, dtype=np.float64).reshape(self.nodes + (3,))
        tgt = np.zeros_like(W) if target is None else np.asarray(target, dtype=np.float64).reshape(W.shape)
        m = np.array(m0, dtype=np.float64).reshape(W.shape)
        if method == DP54:
            c, a, b, _ = dp5_tableau()
            S = 7
        else:
            c, b, S = _RK4_C, _RK4_B, 4
            a = np.zeros((4, 3))
            for s in range(4):
                for j, v in enumerate(_RK4_A[s]):
                    a[s, j] = v
        loss = 0.0
        if include_initial:
            loss += _sample_loss(m, W, tgt)[0]
        # forward with a tape of every stage input
        tape = []
        k1 = self.f(m, plan[0][0]) if (method == DP54 and plan) else None
        if method == DP54 and plan:
            tape0 = (m.copy(), plan[0][0])
        for t, dt, is_sample in plan:
            ys, ks = [], []
            for s in range(S):
                if s == 0:
                    y = m.copy()
                    k = k1 if method == DP54 else self.f(y, t)
                else:
                    y = m + dt * sum(a[s, j] * ks[j] for j in range(s))
                    k = self.f(y, t + c[s] * dt)
                ys.append(y)
                ks.append(k)
            v = ys[-1] if method == DP54 else m + dt * sum(b[s] * ks[s] for s in range(S))
            mn = v.copy()
            if renorm:
                nrm = np.linalg.norm(mn, axis=-1, keepdims=True)
                mn = np.where(nrm > 0, mn / np.where(nrm > 0, nrm, 1.0), mn)
            tape.append((t, dt, is_sample, ys, v, m.copy()))
            if method == DP54:
                k1 = ks[-1]
            m = mn
            if is_sample:
                loss += _sample_loss(m, W, tgt)[0]
        # reverse
        gMs = np.zeros(self.n)
        mbar = np.zeros(W.shape)
        k1bar = np.zeros(W.shape)  # adjoint of the FSAL slope carried into the step after this one
        for t, dt, is_sample, ys, v, m_in in reversed(tape):
            mn = v.copy()
            if renorm:
                nrm = np.linalg.norm(v, axis=-1, keepdims=True)
                mn = np.where(nrm > 0, v / np.where(nrm > 0, nrm, 1.0), v)
            if is_sample:
                mbar = mbar + _sample_loss(mn, W, tgt)[1]
            # through the renormalisation: d(v/|v|)/dv = (I - u u^T)/|v|, symmetric
            if renorm:
                nrm = np.linalg.norm(v, axis=-1, keepdims=True)
                u = np.where(nrm > 0, v / np.where(nrm > 0, nrm, 1.0), 0.0)
                vbar = np.where(nrm > 0, (mbar - u * np.sum(u * mbar, axis=-1, keepdims=True))
                                / np.where(nrm > 0, nrm, 1.0), mbar)
            else:
                vbar = mbar
            kbar = [np.zeros(W.shape) for _ in range(S)]
            ybar = [np.zeros(W.shape) for _ in range(S)]
            new_mbar = np.zeros(W.shape)
            if method == DP54:
                ybar[S - 1] += vbar          # v is the last stage input
                kbar[S - 1] += k1bar         # the last slope is the next step's first slope
            else:
                new_mbar += vbar
                for s in range(S):
                    kbar[s] += dt * b[s] * vbar
            for s in range(S - 1, -1, -1):
                if s > 0 or method == RK4:
                    gm, gs = self.vjp(ys[s], t + c[s] * dt, kbar[s])
                    ybar[s] += gm
                    gMs += gs
                elif s == 0:
                    pass  # the first slope of a Dormand-Prince step is an input (FSAL)
                new_mbar += ybar[s]
                for j in range(s):
                    kbar[j] += dt * a[s, j] * ybar[s]
            mbar = new_mbar
            k1bar = kbar[0] if method == DP54 else np.zeros(W.shape)
        if method == DP54 and plan:
            # the first step's first slope is f(t0, m0)
            m_first, t_first = tape0
            gm, gs = self.vjp(m_first, t_first, k1bar)
            mbar = mbar + gm
            gMs += gs
        if include_initial:
            mbar = mbar + _sample_loss(np.asarray(m0, dtype=np.float64).reshape(W.shape), W, tgt)[1]
        return loss, gMs, mbar
