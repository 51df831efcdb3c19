"""The checkpointed reversal of the RK time integration
(autograd.reverse_steps, binomial schedule), on the CPU with a stand-in mesh
whose step is a small nonlinear map and whose step VJP is that map's exact
transposed Jacobian: the reversed cotangent equals torch.autograd through the
unrolled steps for every snapshot budget, each step is reversed at the state
it started from, the functional's end-of-step callbacks see the trajectory
from the last step to the first, and the recomputed forward steps are the
minimum of Griewank's binomial bound for every length and budget."""
from math import comb

import pytest
import torch

from paper_2210_03523_gb300 import autograd as AG


class StepMesh:
    """q <- q + dt * sin(q) * c (in place); its VJP lam <- lam + dt * cos(q) * c * lam."""

    def __init__(self, n):
        self.c = torch.linspace(0.5, 1.5, n, dtype=torch.float64)
        self.forward_steps = 0

    def rk_step(self, q, g, dt):
        self.forward_steps += 1
        q.add_(dt * torch.sin(q) * self.c)

    def rk_step_vjp(self, q, dt, lam, qinf_adj=None):
        lam.add_(dt * torch.cos(q) * self.c * lam)


def _reference(q0, dt, n, lam, weights=None):
    """torch.autograd through the unrolled steps of the same map"""
    c = torch.linspace(0.5, 1.5, q0.numel(), dtype=torch.float64)
    x = q0.clone().requires_grad_(True)
    q = x
    J = 0.0
    for k in range(n):
        q = q + dt * torch.sin(q) * c
        if weights is not None:
            J = J + (weights[k] * q).sum()
    J = J + (lam * q).sum()
    J.backward()
    return x.grad


@pytest.mark.parametrize("n", [1, 2, 7, 16, 33])
@pytest.mark.parametrize("snapshots", [0, 1, 2, 3, 8])
def test_reverse_matches_autograd_for_every_budget(n, snapshots):
    torch.manual_seed(n)
    q0 = torch.randn(6, dtype=torch.float64)
    lam0 = torch.randn(6, dtype=torch.float64)
    dt = torch.tensor([0.3], dtype=torch.float64)
    mesh = StepMesh(6)
    lam = lam0.clone()
    AG.reverse_steps(mesh, q0, dt, n, lam, snapshots)
    assert torch.allclose(lam, _reference(q0, 0.3, n, lam0), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("snapshots", [0, 2, 8])
def test_end_of_step_callbacks_run_last_step_first(snapshots):
    torch.manual_seed(5)
    n = 11
    q0 = torch.randn(4, dtype=torch.float64)
    dt = torch.tensor([0.2], dtype=torch.float64)
    mesh = StepMesh(4)
    traj = [q0.clone()]
    for _ in range(n):
        traj.append(AG.advance_fixed(mesh, traj[-1], dt, 1))
    weights = [torch.randn(4, dtype=torch.float64) for _ in range(n)]
    seen = []

    def at_end(q, lam):        # a functional sum_k w_k . q_k: its cotangent at the end of step k
        k = len(seen)
        seen.append(q.clone())
        lam.add_(weights[n - 1 - k])
    lam = torch.zeros(4, dtype=torch.float64)
    AG.reverse_steps(mesh, q0, dt, n, lam, snapshots, at_end=at_end)
    assert len(seen) == n
    for k, q in enumerate(seen):   # last step first
        assert torch.allclose(q, traj[n - k], rtol=0, atol=1e-15)
    assert torch.allclose(lam, _reference(q0, 0.2, n, torch.zeros(4, dtype=torch.float64), weights), rtol=1e-13,
                          atol=1e-13)


def _griewank(n, snapshots):
    """The least forward steps that reverse n steps with c = snapshots + 1
    checkpoints (the start state held too): r n - C(c + r, r - 1) for the least
    r with C(c + r, c) >= n (Griewank 1992)."""
    c, r = snapshots + 1, 0
    while comb(c + r, c) < n:
        r += 1
    return r * n - comb(c + r, r - 1) if r else 0


@pytest.mark.parametrize("snapshots", [0, 1, 2, 3, 6, 12])
def test_schedule_meets_the_binomial_bound(snapshots):
    for n in range(1, 130):
        assert AG.reversal_cost(n, snapshots) == _griewank(n, snapshots), n


@pytest.mark.parametrize("n,snapshots", [(64, 0), (64, 1), (64, 2), (64, 6), (400, 12), (37, 3)])
def test_recomputed_steps_are_the_schedules(n, snapshots):
    """the forward steps the reverse sweep actually takes are the schedule's
    count (the last end state supplied by the forward run)"""
    mesh = StepMesh(3)
    lam = torch.ones(3, dtype=torch.float64)
    q0 = torch.zeros(3, dtype=torch.float64)
    dt = torch.tensor([0.1], dtype=torch.float64)
    qn = AG.advance_fixed(StepMesh(3), q0, dt, n)
    AG.reverse_steps(mesh, q0, dt, n, lam, snapshots, at_end=lambda q, l: None, q_end=qn)
    assert mesh.forward_steps == AG.reversal_cost(n, snapshots) == _griewank(n, snapshots)
    if snapshots == 0:
        assert mesh.forward_steps == n * (n - 1) // 2


def test_cylinder_budget_is_far_below_bisection():
    """400 steps with 12 snapshots (the cylinder adjoint): 1080 recomputed
    steps, 2.7 n, against the 1664 of recursive bisection (half the interval
    recomputed at each of its levels)"""
    assert AG.reversal_cost(400, 12) == 1080

    def bisect(n, s):
        if n <= 1:
            return 0
        if s <= 0:
            return n * (n - 1) // 2
        h = n // 2
        return h + bisect(n - h, s - 1) + bisect(h, s)
    assert bisect(400, 12) > 1.5 * AG.reversal_cost(400, 12)
