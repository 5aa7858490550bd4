"""Binomial (revolve) checkpointing of differentiated runs, on the CPU.

revolve_table is the optimal offline checkpointing recursion; it must equal
Griewank's closed form for the fewest forward steps with c + 1 checkpoint
slots (the start state's included): r l - C(c + 1 + r, c + 2), r the least
integer with C(c + 1 + r, c + 1) >= l.  FvRevolveFunction runs its schedule
on a stand-in solver (a fixed linear step on CPU tensors, its transpose as
the VJP): the gradient must equal the one from reversing with every state
stored, bit for bit, with the predicted number of recomputed steps and no
more than `snapshots` states held besides the start state."""
from math import comb

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2306_14011_gb300.autograd import FvRevolveFunction, revolve_table  # noqa: E402


def test_table_equals_the_binomial_closed_form():
    cost, _ = revolve_table(300, 10)
    for c in range(1, 11):
        for l in range(2, 301):
            r = 0
            while comb(c + 1 + r, c + 1) < l:
                r += 1
            assert cost[c][l] == r * l - comb(c + 1 + r, c + 2), (c, l)
    ls = np.arange(301)
    assert np.array_equal(cost[0][1:], ls[1:] * (ls[1:] - 1) // 2)  # no snapshot: recompute every step
    for l in range(2, 11):
        assert cost[10][l] == l - 1  # enough snapshots: store every state


class LinearSolver:
    """Stand-in for fv.Solver: U <- A U per step (A fixed), VJP lam -> A^T lam;
    counts steps and tracks how many step states are alive."""

    def __init__(self, n, seed):
        g = torch.Generator().manual_seed(seed)
        self.A = torch.randn(n, n, dtype=torch.float64, generator=g) / n ** 0.5 + torch.eye(n, dtype=torch.float64)
        self.steps = 0

    def rk_step(self, U, dt):
        U.copy_(self.A @ U)
        self.steps += 1

    def run(self, U, k, dt_fixed=0.0):
        for _ in range(k):
            self.rk_step(U, dt_fixed)

    def rk_step_vjp(self, U, lam, dt, out):
        out.copy_(self.A.T @ lam)
        return out


@pytest.mark.parametrize("nsteps", [1, 2, 3, 7, 40, 157])
@pytest.mark.parametrize("snapshots", [0, 1, 2, 5, 200])
def test_revolve_gradient_is_bitwise_the_stored_states_gradient(nsteps, snapshots):
    S = LinearSolver(6, seed=nsteps)
    x = torch.randn(6, dtype=torch.float64, generator=torch.Generator().manual_seed(1))
    w = torch.randn(6, dtype=torch.float64, generator=torch.Generator().manual_seed(2))
    X0 = x.clone().requires_grad_()
    U = FvRevolveFunction.apply(X0, S, nsteps, 0.1, snapshots)
    forward_steps = S.steps
    assert forward_steps == nsteps
    (w * U).sum().backward()
    # reference: every state kept, VJPs in reverse order (the same operations)
    ref_state = x.clone()
    for _ in range(nsteps):
        ref_state = S.A @ ref_state
    assert torch.equal(U.detach(), ref_state)
    lam = w.clone()
    for _ in range(nsteps):
        lam = S.A.T @ lam
    assert torch.equal(X0.grad, lam)
    cost, split = revolve_table(nsteps, snapshots)
    # recomputation: the table's total minus the advances the forward pass made
    pos, free = 0, snapshots
    while free > 0 and nsteps - pos > 1:
        pos += int(split[free][nsteps - pos])
        free -= 1
    assert S.steps - forward_steps == cost[snapshots][nsteps] - pos


def test_revolve_holds_at_most_the_given_snapshots():
    """The forward pass keeps the start state and at most `snapshots` states;
    the backward pass nests at most `snapshots` reversals, each holding one
    state."""
    n, snapshots = 60, 3
    S = LinearSolver(5, seed=3)
    X0 = torch.randn(5, dtype=torch.float64).requires_grad_()
    U = FvRevolveFunction.apply(X0, S, n, 0.1, snapshots)
    # after the forward pass: the start state plus at most `snapshots` states
    from paper_2306_14011_gb300 import autograd as AG
    fn = U.grad_fn
    states = [s for s in fn.states if s is not None]
    assert len(states) <= snapshots + 1
    peak = {"n": 0, "cur": 0}

    def counting_reverse(orig):
        def wrapped(solver, dt, start, a, b, free, split, lam, out):
            peak["cur"] += 1
            peak["n"] = max(peak["n"], peak["cur"])
            try:
                return orig(solver, dt, start, a, b, free, split, lam, out)
            finally:
                peak["cur"] -= 1
        return wrapped

    orig = AG._reverse
    AG._reverse = counting_reverse(orig)
    try:
        U.sum().backward()
    finally:
        AG._reverse = orig
    # nested reversals each hold one snapshot: never more than `snapshots` deep
    assert 1 <= peak["n"] <= snapshots + 1
    assert X0.grad is not None and torch.isfinite(X0.grad).all()


def test_bad_arguments():
    with pytest.raises(ValueError):
        revolve_table(0, 3)
    with pytest.raises(ValueError):
        revolve_table(5, -1)
    S = LinearSolver(3, seed=0)
    with pytest.raises(ValueError):
        FvRevolveFunction.apply(torch.zeros(3, dtype=torch.float64, requires_grad=True), S, 5, 0.0, 2)
