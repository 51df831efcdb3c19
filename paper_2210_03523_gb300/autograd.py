"""Gradients through the DGSEM residual, the RK3 time integration and the
wall force (drag and lift).

torch.autograd.Function wrappers whose forward passes call dg_residual /
dg_rk_step and whose backward passes call the library's adjoint kernels
(dg_residual_vjp, dg_rk_step_vjp).  The multi-step function does not keep
every state: its reverse sweep stores a bounded number of step states and
recomputes the others (recursive checkpointing: the interval is split in
two, the right half reversed from a snapshot at the split, then the left
half; with no snapshot left, each state is recomputed from the interval's
start).  All arithmetic runs in the library's kernels; this module only
orders the calls.
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


def reverse_steps(mesh, q_l, dt, n, lam, snapshots, at_end=None, qinf_adj=None):
    """lam (the cotangent of the state n steps after q_l) becomes the cotangent of
    q_l, in place.  At most `snapshots` extra states are held at any time.
    at_end(q, lam): called with the state at the end of every step (last step
    first), before that step is reversed, to add a functional's cotangent.
    qinf_adj: accumulates the far-field state's cotangent."""
    if n == 0:
        return lam
    if n == 1:
        if at_end is not None:
            at_end(advance_fixed(mesh, q_l, dt, 1), lam)
        mesh.rk_step_vjp(q_l, dt, lam, qinf_adj)
        return lam
    if snapshots <= 0:
        for k in range(n - 1, -1, -1):
            reverse_steps(mesh, advance_fixed(mesh, q_l, dt, k), dt, 1, lam, 0, at_end, qinf_adj)
        return lam
    half = n // 2
    q_m = advance_fixed(mesh, q_l, dt, half)
    reverse_steps(mesh, q_m, dt, n - half, lam, snapshots - 1, at_end, qinf_adj)
    del q_m
    return reverse_steps(mesh, q_l, dt, half, lam, snapshots, at_end, qinf_adj)


class RKSteps(torch.autograd.Function):
    """n_steps Williamson RK3 steps of fixed size dt (device scalar, not
    differentiated) from q0, with backward through dg_rk_step_vjp under
    recursive checkpointing with `snapshots` stored states."""

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
                  at_end=lambda qe, lm: mesh.wall_force_vjp(qe, lam_f, tag, out=lm, scale=one), qinf_adj=qinf_adj)
    return float(J), lam, qinf_adj


def rk_steps(q0, mesh, dt, n_steps, snapshots=8):
    return RKSteps.apply(q0, mesh, dt, n_steps, snapshots)


def residual(q, mesh):
    return Residual.apply(q, mesh)


__all__ = ["Residual", "RKSteps", "WallForce", "rk_steps", "residual", "wall_force", "time_averaged_force",
           "advance_fixed", "reverse_steps", "dg"]
