"""torch.autograd front end of the discrete adjoint (section "Inverse Micromagnetics").

``llg_loss(mesh, Ms, m0, weight, spec, h=None)`` integrates the LLG equation on ``mesh`` with the cell
Ms map ``Ms``, initial state ``m0`` and (optionally) the uniform applied field ``h`` (A/m, shape (3,))
and returns the sampled quadratic loss
    L = sum_k sum_{n,j} weight_{n,j} (m_{n,j}(t_k) - target_{n,j})^2
as a differentiable torch scalar.  The library computes the loss and its exact discrete gradient in
one call (forward integration with checkpoints, then the adjoint of every accepted step with the step
sizes frozen); ``backward`` hands the stored gradients to autograd.  With ``h`` given, the field is
set on the mesh (frequency and phase from the spec) and dL/dh is returned too, so that field
parameters such as the angles of the paper's inverse problem (section "Inverse Problems") can be
optimised through autograd.

With ``spec.adjoint = "continuous"`` the gradients come from the continuous adjoint-state method
instead (Eq. adjoint_system): a final-time loss, round((t_end - t0) / dt0) classical Runge-Kutta steps
forward, and the adjoint system integrated backwards (nm_adjoint_continuous).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import torch

from . import DP54


@dataclass
class LossSpec:
    """Everything of the integration except the two differentiable inputs (Ms map and m0)."""
    t_end: float
    A: object
    Ku: object = 0.0
    axis: tuple = (0.0, 0.0, 1.0)
    alpha: float = 0.1
    gamma: float = 2.2127614872e5
    target: Optional[np.ndarray] = None
    method: int = DP54
    rtol: float = 1e-5
    atol: float = 1e-5
    dt0: float = 1e-14
    sample_dt: float = 0.0
    include_initial: bool = False
    checkpoint_every: int = 32
    t0: float = 0.0
    h_freq: float = 0.0      # time dependence of the uniform field when h is passed to llg_loss
    h_phase: float = 0.0
    adjoint: str = "discrete"  # or "continuous" (final-time loss, RK4 steps of dt0)
    stats: dict = field(default_factory=dict)


class _LLGLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Ms, m0, h, mesh, weight, spec):
        Ms_h = Ms.detach().to("cpu", torch.float64).numpy()
        m0_h = m0.detach().to("cpu", torch.float64).numpy()
        mesh.set_material(Ms_h, spec.A, spec.Ku, spec.axis, spec.alpha, spec.gamma)
        if h is not None:
            mesh.set_uniform_field(h.detach().to("cpu", torch.float64).numpy(), spec.h_freq, spec.h_phase)
        mesh.set_state(m0_h, spec.t0, spec.dt0)
        if spec.adjoint == "continuous":
            if spec.sample_dt > 0 or spec.include_initial:
                raise ValueError("the continuous adjoint takes a final-time loss (sample_dt = 0, no initial term)")
            n = max(1, int(round((spec.t_end - spec.t0) / spec.dt0)))
            loss, gm0, gMs, gh, _ = mesh.adjoint_continuous(spec.t_end, n, weight, spec.target)
        elif spec.adjoint == "discrete":
            loss, gMs, gm0, n, gh = mesh.adjoint_run(spec.t_end, weight, spec.target, spec.method, spec.rtol,
                                                     spec.atol, spec.dt0, spec.sample_dt, spec.include_initial,
                                                     spec.checkpoint_every, field_grad=True)
        else:
            raise ValueError(f"unknown adjoint {spec.adjoint!r}")
        spec.stats["accepted_steps"] = n
        gh_t = torch.from_numpy(gh).to(h.device, h.dtype) if h is not None else torch.zeros(3)
        ctx.save_for_backward(torch.from_numpy(gMs).to(Ms.device, Ms.dtype),
                              torch.from_numpy(gm0).to(m0.device, m0.dtype), gh_t)
        ctx.has_h = h is not None
        return torch.tensor(loss, dtype=Ms.dtype, device=Ms.device)

    @staticmethod
    def backward(ctx, g):
        gMs, gm0, gh = ctx.saved_tensors
        return g * gMs, g * gm0, (g * gh if ctx.has_h else None), None, None, None


def llg_loss(mesh, Ms: torch.Tensor, m0: torch.Tensor, weight: np.ndarray, spec: LossSpec,
             h: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Differentiable sampled loss of an LLG run (gradients with respect to Ms, m0 and, when given, the
    uniform applied field h)."""
    return _LLGLoss.apply(Ms, m0, h, mesh, weight, spec)
