"""torch.autograd binding of the scheme's reverse mode (hjlo_adjoint).

    u_n = LaxOleinik.apply(u0, P, V, spec)      # spec: Spec(shape, dx, h, W, nsteps, checkpoint_every)

Forward runs nsteps of the scheme (hjlo_run); backward calls hjlo_adjoint,
which recomputes the forward from checkpoints and routes the cotangent back
along the recorded argmins (the discrete optimal path of eq. raslebol).  The
gradients with respect to u0, P (the vector of eq. HPV) and V are returned;
a potential built from coefficients with torch operations gets its
coefficient gradients from torch's own chain rule, or directly from
Plan.project.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import hjlo

__all__ = ["Spec", "LaxOleinik"]


@dataclass(frozen=True)
class Spec:
    shape: tuple
    dx: tuple
    h: float
    W: tuple
    nsteps: int
    checkpoint_every: int = 0


class LaxOleinik(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, P, V, spec: Spec):
        Ph = [float(x) for x in P.detach().cpu().reshape(-1)]
        plan = hjlo.Plan(spec.shape, spec.dx, spec.h, Ph, spec.W)
        u = u0.detach().clone().contiguous()
        plan.run(u, None if V is None else V.detach().contiguous(), spec.nsteps)
        ctx.save_for_backward(u0, P, V if V is not None else torch.empty(0))
        ctx.spec = spec
        ctx.has_V = V is not None
        ctx.plan = plan
        return u

    @staticmethod
    def backward(ctx, grad_un):
        u0, P, V = ctx.saved_tensors
        spec = ctx.spec
        V = V.detach().contiguous() if ctx.has_V else None
        ubar0, Pbar, Vbar, _ = ctx.plan.adjoint(u0.detach().contiguous(), V, spec.nsteps,
                                                grad_un.detach().contiguous(), spec.checkpoint_every,
                                                want_V=ctx.has_V)
        return ubar0, Pbar.to(P.device, P.dtype).reshape(P.shape), Vbar, None
