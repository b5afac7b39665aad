"""Differentiable rollouts: the hand-written discrete adjoint of the step behind
a torch.autograd.Function, with sqrt(N) checkpointing.

``rollout_velocity(solver, force, f0, nsteps)`` advances the state ``f0``
(a storage-layout buffer) by ``nsteps`` steps under the body-acceleration field
``force`` ([2, ny, nx], FP64, CUDA) and returns the final velocity [2, ny, nx]
(FP64).  Its backward pass gives d/d force.  The forward pass keeps one
checkpoint every ``k = ceil(sqrt(nsteps))`` steps; the backward pass walks the
segments in reverse, re-runs each segment forward from its checkpoint while
keeping its k states, and applies the adjoint step (libfdlbm
``fdlbm_adjoint_step``) to them in reverse order.  Memory: about 2 sqrt(N)
states; work: one extra forward pass plus N adjoint steps.
"""
from __future__ import annotations

import math

import torch

from .solver import FDLBM


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, force, solver: FDLBM, f0, nsteps: int):
        solver.set_force(force)
        k = max(1, int(math.ceil(math.sqrt(nsteps))))
        ckpts = []
        solver.load_state(f0)
        done = 0
        while done < nsteps:
            ckpts.append(solver.save_state(solver.new_buffer()))
            n = min(k, nsteps - done)
            solver.step(n)
            done += n
        final = solver.save_state(solver.new_buffer())
        _, ux, uy = solver.moments(device=True)
        ctx.solver, ctx.ckpts, ctx.final, ctx.nsteps, ctx.k = solver, ckpts, final, nsteps, k
        ctx.shape = tuple(force.shape)
        return torch.stack([ux, uy])

    @staticmethod
    def backward(ctx, grad_u):
        s: FDLBM = ctx.solver
        dforce = torch.zeros(ctx.shape, dtype=torch.float64, device=s.device)
        lam = s.new_buffer()
        lam2 = s.new_buffer()
        keep = s.moments_vjp(ctx.final, grad_u, lam, dforce)
        seg = [s.new_buffer() for _ in range(ctx.k)]
        for c in range(len(ctx.ckpts) - 1, -1, -1):
            start = c * ctx.k
            n = min(ctx.k, ctx.nsteps - start)
            s.load_state(ctx.ckpts[c])
            for j in range(n):
                s.save_state(seg[j])
                if j + 1 < n:
                    s.step(1)
            for j in range(n - 1, -1, -1):
                s.adjoint_step(seg[j], lam, lam2, dforce)
                lam, lam2 = lam2, lam
        del keep
        return dforce, None, None, None


def rollout_velocity(solver: FDLBM, force: torch.Tensor, f0: torch.Tensor, nsteps: int):
    """Final velocity after ``nsteps`` steps from ``f0`` under ``force``
    (differentiable with respect to ``force``)."""
    return _Rollout.apply(force, solver, f0, nsteps)
