"""Gradients through the DGSEM residual and the RK3 time integration.

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


def reverse_steps(mesh, q_l, dt, n, lam, snapshots):
    """lam (the cotangent of the state n steps after q_l) becomes the cotangent of
    q_l, in place.  At most `snapshots` extra states are held at any time."""
    if n == 0:
        return lam
    if n == 1:
        mesh.rk_step_vjp(q_l, dt, lam)
        return lam
    if snapshots <= 0:
        for k in range(n - 1, -1, -1):
            mesh.rk_step_vjp(advance_fixed(mesh, q_l, dt, k), dt, lam)
        return lam
    half = n // 2
    q_m = advance_fixed(mesh, q_l, dt, half)
    reverse_steps(mesh, q_m, dt, n - half, lam, snapshots - 1)
    del q_m
    return reverse_steps(mesh, q_l, dt, half, lam, snapshots)


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


def rk_steps(q0, mesh, dt, n_steps, snapshots=8):
    return RKSteps.apply(q0, mesh, dt, n_steps, snapshots)


def residual(q, mesh):
    return Residual.apply(q, mesh)


__all__ = ["Residual", "RKSteps", "rk_steps", "residual", "advance_fixed", "reverse_steps", "dg"]
