"""Continuous adjoint-state gradients for the FP64 oracle (section "Inverse Micromagnetics",
Eqs. adjoint_forward, adjoint_objective and adjoint_system of the paper).

TEST INFRASTRUCTURE ONLY, under the same rule as the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it.  It never imports the
CUDA library.

The forward problem dm/dt = f(t, m) is the LLG right-hand side of the oracle.  The objective is
L = sum W (m(T) - target)^2.  The adjoint system

    dm/dt = f(t, m),   da/dt = -(df/dm)^T a,   du/dt = -(df/dtheta)^T a,
    m(T) = m_output,   a(T) = dL/dm(T),        u(T) = 0,

is integrated backwards from T to t0 with classical Runge-Kutta steps.  u(t0) is the gradient with
respect to the design variables; here theta is the uniform applied field h (3 components), and
a(t0) is the gradient with respect to the initial magnetisation.

Everything is dense and small on purpose: the field Jacobian is assembled column by column from the
oracle's linear field (exchange, anisotropy and demag are linear in m; the Zeeman field does not depend
on m), and the LLG Jacobian follows from the product rule per node:

    f = -g' (m x H + alpha m x (m x H)),  g' = gamma / (1 + alpha^2)
    df/dH = -g' ([m]x + alpha [m]x [m]x)
    df/dm |_H = -g' (-[H]x + alpha ((m . H) I + m H^T - 2 H m^T))
    df/dm = df/dm |_H + df/dH J_h

with zero rows on nodes without magnetic material.
"""
from __future__ import annotations

import numpy as np

from . import ALL, ZEE


def _crossmat(v):
    """[v]x for a stack of 3-vectors: (..., 3) -> (..., 3, 3), [v]x w = v x w."""
    z = np.zeros(v.shape[:-1])
    return np.stack([np.stack([z, -v[..., 2], v[..., 1]], -1),
                     np.stack([v[..., 2], z, -v[..., 0]], -1),
                     np.stack([-v[..., 1], v[..., 0], z], -1)], -2)


class ContinuousAdjoint:
    """Dense continuous-adjoint machinery of one oracle mesh and term set."""

    def __init__(self, mesh, terms=ALL):
        self.mesh = mesh
        self.terms = terms
        self.nodes = mesh.nodes
        self.N = int(np.prod(self.nodes))
        self.magnetic = mesh.mass().reshape(-1) > 0.0
        self.gp = mesh.gamma / (1.0 + mesh.alpha ** 2)
        self.alpha = mesh.alpha
        lin = terms & ~ZEE
        # J_h: column j is the linear field of the unit vector e_j (flattened node-major, component last)
        n3 = 3 * self.N
        J = np.zeros((n3, n3))
        e = np.zeros(n3)
        for j in range(n3):
            e[j] = 1.0
            J[:, j] = mesh.h_eff(e.reshape(self.nodes + (3,)), lin, 0.0).reshape(-1)
            e[j] = 0.0
        self.Jh = J

    def field(self, m, t):
        """H(m, t) = J_h m + h_Zeeman(t), flattened."""
        h = self.Jh @ m.reshape(-1)
        if self.terms & ZEE:
            h = h + self.mesh.h_eff(np.zeros(self.nodes + (3,)), ZEE, t).reshape(-1)
        return h

    def blocks(self, m, t):
        """Per-node 3x3 blocks df/dm|_H and df/dH (zero on non-magnetic nodes)."""
        mm = m.reshape(-1, 3)
        H = self.field(m, t).reshape(-1, 3)
        Cm, CH = _crossmat(mm), _crossmat(H)
        I = np.eye(3)
        mH = np.einsum("ni,ni->n", mm, H)
        Dm = -self.gp * (-CH + self.alpha * (mH[:, None, None] * I + np.einsum("ni,nj->nij", mm, H)
                                            - 2.0 * np.einsum("ni,nj->nij", H, mm)))
        DH = -self.gp * (Cm + self.alpha * np.einsum("nij,njk->nik", Cm, Cm))
        Dm[~self.magnetic] = 0.0
        DH[~self.magnetic] = 0.0
        return Dm, DH

    def rhs(self, m, t):
        return self.mesh.llg_rhs(m.reshape(self.nodes + (3,)), self.terms, t).reshape(-1)

    def jacobian(self, m, t):
        """Dense df/dm (3N x 3N)."""
        Dm, DH = self.blocks(m, t)
        n3 = 3 * self.N
        J = np.zeros((n3, n3))
        for n in range(self.N):
            J[3 * n:3 * n + 3, 3 * n:3 * n + 3] += Dm[n]
        DHJ = np.zeros((n3, n3))
        for n in range(self.N):
            DHJ[3 * n:3 * n + 3, :] = DH[n] @ self.Jh[3 * n:3 * n + 3, :]
        return J + DHJ

    def adjoint_rhs(self, m, a, t, s_t):
        """(-(df/dm)^T a, -(df/dh)^T a) at (m, t); s_t is the time factor of the uniform field."""
        Dm, DH = self.blocks(m, t)
        ka = -(self.jacobian(m, t).T @ a)
        aa = a.reshape(-1, 3)
        kh = -s_t * np.einsum("nji,nj->i", DH, aa)  # sum over magnetic nodes of (df_n/dH_n)^T a_n
        return ka, kh

    def run(self, m0, t0, t_end, n_steps, W, target=None, renorm=True, h_freq=0.0, h_phase=0.0):
        """Forward RK4 to t_end, then the backward adjoint system.  Returns (loss, grad_m0, grad_h, m0_rec)."""
        mesh, terms = self.mesh, self.terms
        h = (t_end - t0) / n_steps
        m = np.asarray(m0, dtype=np.float64).reshape(self.nodes + (3,)).copy()
        t = t0
        for _ in range(n_steps):
            m = mesh.rk4_step(m, t, h, terms, renorm)
            t += h
        W = np.asarray(W, dtype=np.float64).reshape(-1)
        tgt = np.zeros_like(W) if target is None else np.asarray(target, dtype=np.float64).reshape(-1)
        mT = m.reshape(-1)
        loss = float(np.sum(W * (mT - tgt) ** 2))
        a = 2.0 * W * (mT - tgt)
        u = np.zeros(3)
        mb = mT.copy()
        hb = -h
        sfac = (lambda tt: 1.0) if h_freq == 0.0 else (lambda tt: np.sin(2.0 * np.pi * h_freq * tt + h_phase))
        c = (0.0, 0.5, 0.5, 1.0)
        A = ((), (0.5,), (0.0, 0.5), (0.0, 0.0, 1.0))
        b = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)
        for k in range(n_steps):
            tk = t_end - k * h
            km, ka, ku = [], [], []
            for s in range(4):
                ys = mb + hb * sum(A[s][j] * km[j] for j in range(s)) if s else mb.copy()
                as_ = a + hb * sum(A[s][j] * ka[j] for j in range(s)) if s else a.copy()
                ts = tk + c[s] * hb
                km.append(self.rhs(ys, ts))
                kas, khs = self.adjoint_rhs(ys, as_, ts, sfac(ts))
                ka.append(kas)
                ku.append(khs)
            mb = mb + hb * sum(b[s] * km[s] for s in range(4))
            if renorm:
                mm = mb.reshape(-1, 3)
                nrm = np.linalg.norm(mm, axis=1)
                mm[nrm > 0] /= nrm[nrm > 0, None]
            a = a + hb * sum(b[s] * ka[s] for s in range(4))
            u = u + hb * sum(b[s] * ku[s] for s in range(4))
        return loss, a.reshape(self.nodes + (3,)), u, mb.reshape(self.nodes + (3,))
