"""torch.autograd wrappers of the pressure solve, the projection step and
their hand-written adjoints.

Argument marshalling only: the forwards call ``ism_solve`` / ``proj_step``
and the backwards ``ism_solve`` (the solve is symmetric) /
``proj_step_adjoint`` of the CUDA library (``include/ism.h``); no derivative
is taken by torch.  ``rollout_grad`` calls the library's checkpointed rollout,
which runs the whole forward/reverse sweep natively.
"""
from __future__ import annotations

import torch

from . import ism


class IsmSolve(torch.autograd.Function):
    """p = S(rhs): the ISM pressure solve of A_f p = rhs (Sec. 3.4) to `tol`,
    with the mean of rhs removed and p of zero mean when every face is
    Neumann, i.e. S = Pi A_f^+ Pi with Pi the mean projector.  S is
    symmetric, so the backward pass is the same solve applied to the
    incoming gradient (the solver's iterations are not differentiated)."""

    @staticmethod
    def forward(fctx, ctx, rhs, tol, max_cycles):
        p = torch.zeros_like(rhs, dtype=torch.float64)
        ism.check(ism.ism_solve(ctx, rhs.detach().to(torch.float64).contiguous(), p, tol, max_cycles)[0],
                  "ism_solve")
        fctx.args = (ctx, float(tol), int(max_cycles))
        return p

    @staticmethod
    def backward(fctx, gp):
        ctx, tol, max_cycles = fctx.args
        g = torch.zeros_like(gp, dtype=torch.float64)
        ism.check(ism.ism_solve(ctx, gp.detach().to(torch.float64).contiguous(), g, tol, max_cycles)[0],
                  "ism_solve (adjoint)")
        return None, g, None, None


def solve(ctx, rhs, tol=1e-8, max_cycles=100000):
    """Differentiable pressure solve (FP64 in and out)."""
    return IsmSolve.apply(ctx, rhs, tol, max_cycles)


class ProjStep(torch.autograd.Function):
    """(u, v, p) -> (u', v', p') of one projection step (Sec. 2.2-2.3) on the
    flow set up in the context; the inputs are not modified."""

    @staticmethod
    def forward(fctx, ctx, u, v, p, dt, nu):
        uo, vo, po = u.detach().clone(), v.detach().clone(), p.detach().clone()
        ism.check(ism.proj_step(ctx, uo, vo, po, dt, nu), "proj_step")
        fctx.save_for_backward(u, v)
        fctx.args = (ctx, float(dt), float(nu))
        return uo, vo, po

    @staticmethod
    def backward(fctx, gu, gv, gp):
        u, v = fctx.saved_tensors
        ctx, dt, nu = fctx.args
        outs = []
        for g, like in ((gu, u), (gv, v), (gp, None)):
            if g is None:
                shape = like.shape if like is not None else (ctx.ny, ctx.nx)
                g = torch.zeros(shape, dtype=torch.float32, device=u.device)
            outs.append(g.detach().to(torch.float32).contiguous().clone())
        ism.check(ism.proj_step_adjoint(ctx, u.detach(), v.detach(), dt, nu, *outs),
                  "proj_step_adjoint")
        return (None, *outs, None, None)


def proj_step(ctx, u, v, p, dt, nu):
    """Differentiable projection step."""
    return ProjStep.apply(ctx, u, v, p, dt, nu)


def rollout_grad(ctx, u0, v0, p0, dt, nu, steps, every=20):
    """Final enstrophy of a `steps`-step rollout and its gradient with respect
    to (u0, v0, p0), by the library's checkpointed reverse sweep."""
    gu, gv, gp = torch.empty_like(u0), torch.empty_like(v0), torch.empty_like(p0)
    s, loss = ism.proj_rollout_grad(ctx, u0, v0, p0, dt, nu, steps, every, gu, gv, gp)
    ism.check(s, "proj_rollout_grad")
    return loss, gu, gv, gp


def rollout_loss(ctx, u0, v0, p0, dt, nu, steps):
    """Final enstrophy of a `steps`-step rollout (forward only)."""
    s, loss = ism.proj_rollout_grad(ctx, u0, v0, p0, dt, nu, steps, 1)
    ism.check(s, "proj_rollout_grad")
    return loss
