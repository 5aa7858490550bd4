"""Gradients through the solver: torch.autograd.Function wrappers over libfv.

FvRunFunction.apply(U0, solver, nsteps, dt, every) advances U0 by nsteps
SSP-RK3 steps with the step held at dt and differentiates through them with
the discrete adjoint (fv_adjoint_vjp, one RK-step VJP per step in reverse).
Memory is bounded by two-level checkpointing: the forward pass keeps the
state every `every` steps; the backward pass re-runs each segment from its
checkpoint, keeping that segment's step states, then reverses it.  Forward
work is about doubled; stored states are nsteps/every + every.

FvResidualFunction.apply(U, solver) is R_h(U) (Eq. (5)) with its VJP, and
FvStepFunction.apply(U, solver, dt) one SSP-RK3 step with the step held at dt
(Eq. (4)) with its VJP, for composing steps with other torch operations.
Everything runs in the library's kernels; torch only holds the tensors.
"""
from __future__ import annotations

import torch

from . import fv


class FvResidualFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, solver):
        ctx.solver = solver
        ctx.save_for_backward(U)
        return solver.residual(U.detach().contiguous())

    @staticmethod
    def backward(ctx, gR):
        (U,) = ctx.saved_tensors
        return ctx.solver.residual_vjp(U.detach().contiguous(), gR.contiguous()), None


class FvStepFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, solver, dt: float):
        if not dt > 0.0:
            raise ValueError("a differentiated step needs a fixed step dt > 0")
        ctx.solver, ctx.dt = solver, dt
        ctx.save_for_backward(U)
        X = U.detach().contiguous().clone()
        solver.rk_step(X, dt)
        return X

    @staticmethod
    def backward(ctx, gU):
        (U,) = ctx.saved_tensors
        return ctx.solver.rk_step_vjp(U.detach().contiguous(), gU.contiguous(), ctx.dt), None, None


class FvRunFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, solver, nsteps: int, dt: float, every: int = 20):
        if not dt > 0.0:
            raise ValueError("differentiated runs need a fixed step dt > 0")
        every = max(1, int(every))
        U = U0.detach().contiguous().clone()
        ckpts = []
        done = 0
        while done < nsteps:
            k = min(every, nsteps - done)
            ckpts.append(U.clone())
            solver.run(U, k, dt_fixed=dt)
            done += k
        ctx.solver, ctx.nsteps, ctx.dt, ctx.every = solver, nsteps, dt, every
        ctx.ckpts = ckpts
        return U

    @staticmethod
    def backward(ctx, gU):
        solver, dt, every = ctx.solver, ctx.dt, ctx.every
        lam = gU.contiguous().clone()
        out = torch.empty_like(lam)
        for seg in range(len(ctx.ckpts) - 1, -1, -1):
            start = seg * every
            k = min(every, ctx.nsteps - start)
            states = [ctx.ckpts[seg]]
            X = ctx.ckpts[seg].clone()
            for _ in range(k - 1):
                solver.rk_step(X, dt)
                states.append(X.clone())
            for s in range(k - 1, -1, -1):
                fv.fv_adjoint_vjp(solver.ctx, fv.FV_VJP_RKSTEP, states[s], lam, dt, out)
                lam, out = out, lam
        ctx.ckpts = None
        return lam, None, None, None, None


def kinetic_energy(U, grid):
    """J = sum over cells of (m_x^2 + m_y^2 [+ m_z^2]) / (2 rho) * |Omega|."""
    vol = 1.0
    for d in range(grid.dim):
        vol *= grid.length[d] / grid.n[d]
    rho = U[0]
    m2 = sum(U[1 + d] ** 2 for d in range(grid.dim))
    return (0.5 * m2 / rho).sum() * vol
