"""Gradients through the solver: torch.autograd.Function wrappers over libfv.

FvRunFunction.apply(U0, solver, nsteps, dt, every) advances U0 by nsteps
SSP-RK3 steps with the step held at dt and differentiates through them with
the discrete adjoint (fv_adjoint_vjp, one RK-step VJP per step in reverse).
Memory is bounded by two-level checkpointing: the forward pass keeps the
state every `every` steps; the backward pass re-runs each segment from its
checkpoint, keeping that segment's step states, then reverses it.  Forward
work is about doubled; stored states are nsteps/every + every.  With
keep_stages (the default, a sixth argument) the re-run also keeps each
step's two RK stage states (fv_rk_step_stages), so the step VJPs
(fv_adjoint_vjp_stages) do not recompute them: two stage kernels fewer per
step for 2 x every more stored states, the same gradient bit for bit.

FvRevolveFunction.apply(U0, solver, nsteps, dt, snapshots) differentiates the
same run with at most `snapshots` stored states besides U0, placed by the
optimal offline (binomial) checkpointing schedule of Griewank's revolve: the
fewest recomputed steps for that memory (revolve_table).

FvResidualFunction.apply(U, solver) is R_h(U) (Eq. (5)) with its VJP, and
FvStepFunction.apply(U, solver, dt) one SSP-RK3 step with the step held at dt
(Eq. (4)) with its VJP, for composing steps with other torch operations.
Everything runs in the library's kernels; torch only holds the tensors.
"""
from __future__ import annotations

import functools

import numpy as np
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
    def forward(ctx, U0, solver, nsteps: int, dt: float, every: int = 20, keep_stages: bool = True):
        if not dt > 0.0:
            raise ValueError("differentiated runs need a fixed step dt > 0")
        every = max(1, int(every))
        ctx.keep_stages = bool(keep_stages) and hasattr(solver, "rk_step_stages")
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
            if ctx.keep_stages:
                # recompute the segment keeping every step's stage states, so
                # the step VJPs need not recompute them (the same values)
                stages = []
                for s in range(k):
                    U1, U2 = torch.empty_like(X), torch.empty_like(X)
                    solver.rk_step_stages(X, dt, U1, U2)
                    stages.append((U1, U2))
                    if s + 1 < k:
                        states.append(X.clone())
                for s in range(k - 1, -1, -1):
                    solver.rk_step_vjp_stages(states[s], stages[s][0], stages[s][1], lam, dt, out)
                    lam, out = out, lam
                    stages[s] = None
                continue
            for _ in range(k - 1):
                solver.rk_step(X, dt)
                states.append(X.clone())
            for s in range(k - 1, -1, -1):
                fv.fv_adjoint_vjp(solver.ctx, fv.FV_VJP_RKSTEP, states[s], lam, dt, out)
                lam, out = out, lam
        ctx.ckpts = None
        return lam, None, None, None, None, None


@functools.lru_cache(maxsize=16)
def revolve_table(nsteps: int, snapshots: int):
    """Optimal offline checkpointing of `nsteps` steps reversed from a stored
    start state with `snapshots` further states (binomial checkpointing,
    Griewank 1992; Griewank and Walther's revolve).  Returns (cost, split),
    int64 arrays of shape (snapshots + 1, nsteps + 1): cost[c][l] is the
    fewest forward steps that reverse l steps with c free snapshots, split[c][l]
    the steps to advance before storing the next state:
        cost[c][l] = min over 0 < m < l of  m + cost[c-1][l-m] + cost[c][m],
        cost[c][1] = 0,  cost[0][l] = l (l - 1) / 2  (recompute every step)."""
    n, C = int(nsteps), int(snapshots)
    if n < 1 or C < 0:
        raise ValueError("need nsteps >= 1 and snapshots >= 0")
    ls = np.arange(n + 1, dtype=np.int64)
    cost = np.zeros((C + 1, n + 1), dtype=np.int64)
    split = np.zeros((C + 1, n + 1), dtype=np.int64)
    cost[0] = np.maximum(ls * (ls - 1) // 2, 0)
    for c in range(1, C + 1):
        for l in range(2, n + 1):
            m = ls[1:l]
            tot = m + cost[c - 1][l - m] + cost[c][m]
            j = int(np.argmin(tot))
            cost[c][l] = tot[j]
            split[c][l] = m[j]
    cost.setflags(write=False)
    split.setflags(write=False)
    return cost, split


def _reverse(solver, dt, start, a, b, free, split, lam, out):
    """Reverse steps a..b-1 given the state at step a (`start`, unchanged):
    on entry lam is the cotangent of the state at b, on return the first of
    the returned pair is that of the state at a (the second is scratch)."""
    while b > a:
        if b - a == 1:
            solver.rk_step_vjp(start, lam, dt, out)
            return out, lam
        if free == 0:  # no snapshot left: recompute each step from `start`
            X = torch.empty_like(start)
            for j in range(b - 1, a - 1, -1):
                X.copy_(start)
                for _ in range(j - a):
                    solver.rk_step(X, dt)
                solver.rk_step_vjp(X, lam, dt, out)
                lam, out = out, lam
            return lam, out
        m = int(split[free][b - a])
        S = start.clone()
        for _ in range(m):
            solver.rk_step(S, dt)
        lam, out = _reverse(solver, dt, S, a + m, b, free - 1, split, lam, out)
        del S
        b = a + m  # the left part keeps the same number of free snapshots
    return lam, out


class FvRevolveFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, solver, nsteps: int, dt: float, snapshots: int = 20):
        if not dt > 0.0:
            raise ValueError("differentiated runs need a fixed step dt > 0")
        nsteps, snapshots = int(nsteps), int(snapshots)
        _, split = revolve_table(max(1, nsteps), snapshots)
        U = U0.detach().contiguous().clone()
        # the schedule's first advances: from step 0, store a state after
        # split[c][remaining] steps, c = snapshots, snapshots - 1, ...
        pos, states = [0], [U0.detach().contiguous().clone()]  # a copy: U0 may change before backward
        free = snapshots
        while free > 0 and nsteps - pos[-1] > 1:
            m = int(split[free][nsteps - pos[-1]])
            solver.run(U, m, dt_fixed=dt)
            pos.append(pos[-1] + m)
            states.append(U.clone())
            free -= 1
        solver.run(U, nsteps - pos[-1], dt_fixed=dt)
        ctx.solver, ctx.nsteps, ctx.dt, ctx.snapshots = solver, nsteps, dt, snapshots
        ctx.pos, ctx.states = pos, states
        return U

    @staticmethod
    def backward(ctx, gU):
        solver, dt, n, C = ctx.solver, ctx.dt, ctx.nsteps, ctx.snapshots
        _, split = revolve_table(max(1, n), C)
        pos, states = ctx.pos, ctx.states
        lam = gU.contiguous().clone()
        out = torch.empty_like(lam)
        k = len(pos) - 1
        if n > 0:
            lam, out = _reverse(solver, dt, states[k], pos[k], n, C - k, split, lam, out)
        for i in range(k - 1, -1, -1):
            states[i + 1] = None  # its snapshot is free again
            lam, out = _reverse(solver, dt, states[i], pos[i], pos[i + 1], C - i, split, lam, out)
        ctx.states = None
        return lam, None, None, None, None


def kinetic_energy(U, grid):
    """J = sum over cells of (m_x^2 + m_y^2 [+ m_z^2]) / (2 rho) * |Omega|."""
    vol = 1.0
    for d in range(grid.dim):
        vol *= grid.length[d] / grid.n[d]
    rho = U[0]
    m2 = sum(U[1 + d] ** 2 for d in range(grid.dim))
    return (0.5 * m2 / rho).sum() * vol
