"""Differentiable rollouts: the hand-written discrete adjoint of the step behind
torch.autograd.Functions, with sqrt(N) checkpointing.

``rollout_velocity(solver, force, f0, nsteps)`` advances the state ``f0``
(a storage-layout buffer) by ``nsteps`` steps under the body-acceleration field
``force`` ([2, ny, nx], FP64, CUDA) and returns the final velocity [2, ny, nx]
(FP64).  Its backward pass gives d/d force.
``rollout_velocity_from_fields(solver, force, rho, ux, uy, nsteps)`` starts
from the fields instead (f = f^eq of Eq. 3.2, f~ = f - (dt/2) F_i by Eq. 2.19
under ``force``), and its backward pass
also gives d/d rho, d/d ux and d/d uy (libfdlbm ``fdlbm_init_vjp``), so that
an initial velocity (or vorticity, through a differentiable map to u) can be
recovered as well as a force.

The forward pass keeps one checkpoint every ``k = ceil(sqrt(nsteps))`` steps;
the backward pass walks the segments in reverse, re-runs each segment forward
from its checkpoint while keeping its k states, and applies the adjoint step
(libfdlbm ``fdlbm_adjoint_step``) to them in reverse order.  Memory: about
2 sqrt(N) states; work: one extra forward pass plus N adjoint steps.
"""
from __future__ import annotations

import math

import torch

from .solver import FDLBM


def _forward(solver: FDLBM, force, nsteps: int):
    """Run nsteps from the solver's current state under the force already set,
    keeping the checkpoints."""
    k = max(1, int(math.ceil(math.sqrt(nsteps))))
    ckpts = []
    done = 0
    while done < nsteps:
        ckpts.append(solver.save_state(solver.new_buffer()))
        n = min(k, nsteps - done)
        solver.step(n)
        done += n
    final = solver.save_state(solver.new_buffer())
    _, ux, uy = solver.moments(device=True)
    return ckpts, final, k, torch.stack([ux, uy])


def _reverse(s: FDLBM, ckpts, final, nsteps: int, k: int, grad_u, shape):
    """The adjoint sweep: (d/d force, cotangent of the initial state)."""
    dforce = torch.zeros(shape, dtype=torch.float64, device=s.device)
    lam = s.new_buffer()
    lam2 = s.new_buffer()
    keep = s.moments_vjp(final, grad_u, lam, dforce)
    seg = [s.new_buffer() for _ in range(k)]
    for c in range(len(ckpts) - 1, -1, -1):
        start = c * k
        n = min(k, nsteps - start)
        s.load_state(ckpts[c])
        for j in range(n):
            s.save_state(seg[j])
            if j + 1 < n:
                s.step(1)
        for j in range(n - 1, -1, -1):
            s.adjoint_step(seg[j], lam, lam2, dforce)
            lam, lam2 = lam2, lam
    del keep
    return dforce, lam


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, force, solver: FDLBM, f0, nsteps: int):
        solver.load_state(f0)
        solver.set_force(force)
        ckpts, final, k, u = _forward(solver, force, nsteps)
        ctx.solver, ctx.ckpts, ctx.final, ctx.nsteps, ctx.k = solver, ckpts, final, nsteps, k
        ctx.shape = tuple(force.shape)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        dforce, _ = _reverse(ctx.solver, ctx.ckpts, ctx.final, ctx.nsteps, ctx.k, grad_u, ctx.shape)
        return dforce, None, None, None


class _RolloutFields(torch.autograd.Function):
    @staticmethod
    def forward(ctx, force, rho, ux, uy, solver: FDLBM, nsteps: int):
        fields = [t.detach().to(torch.float64).contiguous() for t in (rho, ux, uy)]
        # the force first: the initial state carries -(dt/2) F_i (Eq. 2.19)
        solver.set_force(force)
        solver.init_fields(*fields)
        ckpts, final, k, u = _forward(solver, force, nsteps)
        ctx.solver, ctx.ckpts, ctx.final, ctx.nsteps, ctx.k = solver, ckpts, final, nsteps, k
        ctx.shape = tuple(force.shape)
        ctx.fields = fields
        return u

    @staticmethod
    def backward(ctx, grad_u):
        s: FDLBM = ctx.solver
        dforce, lam0 = _reverse(s, ctx.ckpts, ctx.final, ctx.nsteps, ctx.k, grad_u, ctx.shape)
        drho, dux, duy = (torch.zeros_like(f) for f in ctx.fields)
        s.init_vjp(*ctx.fields, lam0, drho, dux, duy, dforce)
        s.sync()
        return dforce, drho, dux, duy, None, None


def rollout_velocity(solver: FDLBM, force: torch.Tensor, f0: torch.Tensor, nsteps: int):
    """Final velocity after ``nsteps`` steps from ``f0`` under ``force``
    (differentiable with respect to ``force``)."""
    return _Rollout.apply(force, solver, f0, nsteps)


def rollout_velocity_from_fields(solver: FDLBM, force: torch.Tensor, rho: torch.Tensor,
                                 ux: torch.Tensor, uy: torch.Tensor, nsteps: int):
    """Final velocity after ``nsteps`` steps from the equilibrium of (rho, ux,
    uy) ([ny, nx] CUDA tensors) under ``force`` (differentiable with respect to
    ``force``, ``rho``, ``ux`` and ``uy``)."""
    return _RolloutFields.apply(force, rho, ux, uy, solver, nsteps)
