"""Differentiable rollout: n fixed-dt TVD-RK3 steps of the GPU solver as a
torch.autograd.Function (the AD-through-the-solver use of §6).

The forward pass advances the library's state with jxf_step and keeps a
checkpoint every ``ckpt`` steps; the backward pass walks the segments in
reverse, recomputes each segment's states from its checkpoint with the same
steps, and applies the hand-written step adjoint (jxf_step_vjp) step by step.
Memory: (n/ckpt + ckpt) states.
"""
from __future__ import annotations

import torch


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, solver, nsteps: int, dt: float, ckpt: int):
        ckpts = []
        solver.set_state(U0.detach().contiguous())
        for k in range(nsteps):
            if k % ckpt == 0:
                ckpts.append(solver.state())
            solver.step(1, sync=False)
        UT = solver.state()
        ctx.solver, ctx.nsteps, ctx.dt, ctx.ckpt, ctx.ckpts = solver, nsteps, dt, ckpt, ckpts
        return UT

    @staticmethod
    def backward(ctx, gUT):
        s, n, dt, ck = ctx.solver, ctx.nsteps, ctx.dt, ctx.ckpt
        Ub = gUT.contiguous().to(s.dtype)
        for seg in reversed(range(len(ctx.ckpts))):
            start = seg * ck
            stop = min(start + ck, n)
            s.set_state(ctx.ckpts[seg])
            states = [ctx.ckpts[seg]]
            for _ in range(start, stop - 1):
                s.step(1, sync=False)
                states.append(s.state())
            for k in reversed(range(stop - start)):
                Ub = s.step_vjp(states[k], dt, Ub)
        ctx.ckpts = None
        return Ub, None, None, None, None


def rollout(U0, solver, nsteps: int, dt: float, ckpt: int = 100):
    """U(n) from U(0) through n fixed-dt RK3 steps (differentiable in U0).
    ``solver`` must be created with fixed_dt = dt and t_end = 0."""
    return Rollout.apply(U0, solver, nsteps, dt, ckpt)
