"""Gradients through the DGSEM residual, the RK3 time integration and the
wall force (drag and lift).

torch.autograd.Function wrappers whose forward passes call dg_residual /
dg_rk_step and whose backward passes call the library's adjoint kernels
(dg_residual_vjp, dg_rk_step_vjp).  The multi-step function does not keep
every state: its reverse sweep holds a bounded number of step states and
recomputes the others on the binomial checkpointing schedule (Griewank,
"Achieving logarithmic growth of temporal and spatial complexity in reverse
automatic differentiation", 1992; the schedule of the revolve algorithm):
with the start state and s snapshots, c = s + 1 checkpoints, reversing n
steps recomputes the least number of forward steps, r n - C(c + r, r - 1)
for the least r with C(c + r, c) >= n.  All arithmetic runs in the library's
kernels; this module only orders the calls.
"""
from __future__ import annotations

import torch

from . import dg


class Residual(torch.autograd.Function):
    """R(q) with backward (dR/dq)^T g."""

    @staticmethod
    def forward(ctx, q, mesh):
        ctx.mesh = mesh
        ctx.save_for_backward(q)
        return mesh.residual(q.contiguous())

    @staticmethod
    def backward(ctx, g):
        (q,) = ctx.saved_tensors
        return ctx.mesh.residual_vjp(q.contiguous(), g.contiguous()), None


def advance_fixed(mesh, q, dt, n):
    """n RK3 steps of the fixed size dt (a device scalar) from q; returns a new tensor."""
    q = q.clone()
    g = torch.zeros_like(q)
    for _ in range(n):
        mesh.rk_step(q, g, dt)
    return q


_SCHEDULE = {}


def _schedule(n, snapshots):
    """(cost, split) tables of the optimal reversal of up to n steps with up to
    `snapshots` snapshots: cost[s][k] the fewest forward steps that reverse k
    steps holding at most s extra states, split[s][k] where the first snapshot
    goes (0: none, every state recomputed from the start).  The recurrence:
    reversing k > 1 steps from a held start state, advance m steps and hold
    the state there, reverse the last k - m steps with s - 1 snapshots, then
    the first m with s: cost(k, s) = min_m m + cost(k - m, s - 1) + cost(m, s);
    with no snapshot each of the k states is recomputed from the start,
    cost(k, 0) = k (k - 1) / 2; one step costs none."""
    key = (n, snapshots)
    if key in _SCHEDULE:
        return _SCHEDULE[key]
    import numpy as np
    big = np.iinfo(np.int64).max // 4
    cost = np.zeros((snapshots + 1, n + 1), dtype=np.int64)
    split = np.zeros((snapshots + 1, n + 1), dtype=np.int64)
    k = np.arange(n + 1)
    cost[0] = k * (k - 1) // 2
    cost[0, 0] = 0
    for s in range(1, snapshots + 1):
        cost[s, :2] = 0
        for kk in range(2, n + 1):
            m = np.arange(1, kk)
            c = m + cost[s - 1, kk - m] + cost[s, m]
            j = int(np.argmin(c))
            cost[s, kk], split[s, kk] = (c[j], m[j]) if c[j] < cost[0, kk] else (cost[0, kk], 0)
    for s in range(snapshots + 1):
        cost[s, cost[s] > big] = big
    _SCHEDULE[key] = (cost, split)
    return cost, split


def reverse_steps(mesh, q_l, dt, n, lam, snapshots, at_end=None, qinf_adj=None, q_end=None):
    """lam (the cotangent of the state n steps after q_l) becomes the cotangent of
    q_l, in place, on the binomial checkpointing schedule with at most
    `snapshots` extra states held at any time.
    at_end(q, lam): adds a functional's cotangent at the end state q of every
    step (last step first), before that step is reversed; the last step's end
    state is q_end when given (the forward run's result), else recomputed.
    qinf_adj: accumulates the far-field state's cotangent."""
    if n == 0:
        return lam
    if at_end is not None:
        at_end(q_end if q_end is not None else advance_fixed(mesh, q_l, dt, n), lam)
    _, split = _schedule(n, max(int(snapshots), 0))
    _reverse(mesh, q_l, dt, n, lam, max(int(snapshots), 0), split, at_end, qinf_adj)
    return lam


def _reverse(mesh, q_l, dt, n, lam, s, split, at_end, qinf_adj):
    """The recursion of reverse_steps: lam holds every contribution at the
    interval's end state; on return it is the cotangent of q_l (without the
    functional's own term at q_l, which the caller adds)."""
    if n == 1:
        mesh.rk_step_vjp(q_l, dt, lam, qinf_adj)
        return
    m = int(split[s, n]) if s > 0 else 0
    if m == 0:            # no snapshot: every step's start state from q_l
        for k in range(n - 1, -1, -1):
            q_k = advance_fixed(mesh, q_l, dt, k) if k else q_l
            mesh.rk_step_vjp(q_k, dt, lam, qinf_adj)
            if k and at_end is not None:
                at_end(q_k, lam)
        return
    q_m = advance_fixed(mesh, q_l, dt, m)
    _reverse(mesh, q_m, dt, n - m, lam, s - 1, split, at_end, qinf_adj)
    if at_end is not None:
        at_end(q_m, lam)
    del q_m
    _reverse(mesh, q_l, dt, m, lam, s, split, at_end, qinf_adj)


def reversal_cost(n, snapshots):
    """Forward steps the reverse sweep of n steps recomputes with the given
    snapshots (at_end's end state supplied)."""
    cost, _ = _schedule(n, max(int(snapshots), 0))
    return int(cost[max(int(snapshots), 0), n])


class RKSteps(torch.autograd.Function):
    """n_steps Williamson RK3 steps of fixed size dt (device scalar, not
    differentiated) from q0, with backward through dg_rk_step_vjp on the
    binomial checkpointing schedule with `snapshots` stored states."""

    @staticmethod
    def forward(ctx, q0, mesh, dt, n_steps, snapshots=8):
        ctx.mesh, ctx.n, ctx.snapshots = mesh, int(n_steps), int(snapshots)
        ctx.save_for_backward(q0, dt)
        return advance_fixed(mesh, q0.contiguous(), dt, ctx.n)

    @staticmethod
    def backward(ctx, g):
        q0, dt = ctx.saved_tensors
        lam = g.contiguous().clone()
        reverse_steps(ctx.mesh, q0.contiguous(), dt, ctx.n, lam, ctx.snapshots)
        return lam, None, None, None, None


class WallForce(torch.autograd.Function):
    """Force of the fluid on the boundary faces of a tag (dg_wall_force), with
    backward dg_wall_force_vjp."""

    @staticmethod
    def forward(ctx, q, mesh, tag=-2):
        ctx.mesh, ctx.tag = mesh, int(tag)
        ctx.save_for_backward(q)
        return mesh.wall_force(q.contiguous(), ctx.tag)

    @staticmethod
    def backward(ctx, g):
        (q,) = ctx.saved_tensors
        return ctx.mesh.wall_force_vjp(q.contiguous(), g.contiguous(), ctx.tag), None, None


def wall_force(q, mesh, tag=-2):
    return WallForce.apply(q, mesh, tag)


def time_averaged_force(mesh, q0, dt, n_steps, direction=(1.0, 0.0, 0.0), tag=-2, snapshots=8):
    """J = (1/n) sum_{k=1..n} d . F(q_k): the force on the boundary faces of a tag
    (the cylinder's wall: d = e_x gives the drag) averaged over n RK3 steps of
    the fixed size dt from q0, and by the discrete adjoint its gradients with
    respect to q0 and to the far-field state q_inf.  Returns (J, dJ/dq0, dJ/dq_inf)."""
    d = torch.tensor(direction, dtype=torch.float64, device=q0.device)
    q = q0.clone()
    g = torch.zeros_like(q)
    J = torch.zeros((), dtype=torch.float64, device=q0.device)
    for _ in range(n_steps):
        mesh.rk_step(q, g, dt)
        J += d @ mesh.wall_force(q, tag)
    J /= n_steps
    lam_f = d / n_steps
    one = torch.ones(1, dtype=torch.float64, device=q0.device)
    lam = torch.zeros_like(q0)
    qinf_adj = torch.zeros(5, dtype=torch.float64, device=q0.device)
    reverse_steps(mesh, q0.contiguous(), dt, n_steps, lam, snapshots,
                  at_end=lambda qe, lm: mesh.wall_force_vjp(qe, lam_f, tag, out=lm, scale=one), qinf_adj=qinf_adj,
                  q_end=q)
    return float(J), lam, qinf_adj


class AveragedForce(torch.autograd.Function):
    """J = (1/n) sum_{k=1..n} d . F(q_k) (time_averaged_force) as a function of the
    initial state q0 and of the far-field state qinf (a 5-vector tensor equal
    to the mesh's q_inf, the handle of its gradient: the mesh's ghost states
    and BR1 q-hat at far-field faces use it).  Backward: dJ/dq0 and dJ/dqinf
    from the discrete adjoint."""

    @staticmethod
    def forward(ctx, q0, qinf, mesh, dt, n_steps, direction=(1.0, 0.0, 0.0), tag=-2, snapshots=12):
        if not torch.equal(qinf.detach().cpu(), torch.tensor(mesh.mi.phys.qinf, dtype=torch.float64)):
            raise ValueError("qinf: must equal the mesh's far-field state")
        J, lam, qinf_adj = time_averaged_force(mesh, q0.detach().contiguous(), dt, int(n_steps), direction, tag,
                                               snapshots)
        ctx.save_for_backward(lam, qinf_adj)
        return torch.tensor(J, dtype=torch.float64, device=q0.device)

    @staticmethod
    def backward(ctx, g):
        lam, qinf_adj = ctx.saved_tensors
        return lam * g, qinf_adj * g, None, None, None, None, None, None


def averaged_force(q0, qinf, mesh, dt, n_steps, direction=(1.0, 0.0, 0.0), tag=-2, snapshots=12):
    return AveragedForce.apply(q0, qinf, mesh, dt, n_steps, direction, tag, snapshots)


def impulsive_start(mesh, qinf, xyz, r_wall=0.5, sharpness=8.0):
    """The initial state of a flow started impulsively from the inflow state
    qinf (a 5-vector tensor, differentiable): at every node the inflow density
    and total energy, and the inflow momentum ramped to rest at the wall by
    d = 1 - exp(-(r^2 - r_wall^2) sharpness), r the distance from the z axis;
    the pressure is the inflow pressure.  xyz: the mesh's node coordinates
    (dg_node_coords layout).  Returns the state in the mesh's layout."""
    off = mesh.offsets()
    dev = qinf.device
    n_el = len(off) - 1
    counts = torch.as_tensor(off[1:] - off[:-1], device=dev)
    # per scalar of the state layout: its variable and its node
    elem = torch.repeat_interleave(torch.arange(n_el, device=dev), 5 * counts)
    start = torch.as_tensor(5 * off[:-1], device=dev)[elem]
    local = torch.arange(5 * int(off[-1]), device=dev) - start
    var = torch.div(local, counts[elem], rounding_mode="floor")
    node = torch.as_tensor(off[:-1], device=dev)[elem] + local - var * counts[elem]
    x = xyz.view(-1)
    xe = torch.repeat_interleave(torch.arange(n_el, device=dev), counts)
    pos = torch.arange(int(off[-1]), device=dev) - torch.as_tensor(off[:-1], device=dev)[xe]
    base = 3 * torch.as_tensor(off[:-1], device=dev)[xe] + pos
    cx, cy = x[base], x[base + counts[xe]]
    d = 1.0 - torch.exp(-(cx * cx + cy * cy - r_wall * r_wall) * sharpness)
    rho, m, E = qinf[0], qinf[1:4], qinf[4]
    ke = 0.5 * (m * m).sum() / rho
    fields = torch.stack([rho.expand_as(d), m[0] * d, m[1] * d, m[2] * d, E - ke * (1.0 - d * d)])   # [5][node]
    return fields[var, node]


def rk_steps(q0, mesh, dt, n_steps, snapshots=8):
    return RKSteps.apply(q0, mesh, dt, n_steps, snapshots)


def residual(q, mesh):
    return Residual.apply(q, mesh)


__all__ = ["Residual", "RKSteps", "WallForce", "AveragedForce", "rk_steps", "residual", "wall_force",
           "time_averaged_force", "averaged_force", "impulsive_start", "advance_fixed", "reverse_steps",
           "reversal_cost", "dg"]
