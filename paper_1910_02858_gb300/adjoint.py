"""Checkpointed discrete adjoint of the LSERK4(5) time integration as a
torch.autograd.Function.

forward(U0) runs nsteps flexi_rk_step calls and keeps U at the start of every
`checkpoint_every`-th step (dU need not be kept: A_1 = 0 makes the first
stage overwrite it).  backward(gU_T) walks the segments in reverse: it
recomputes a segment from its checkpoint with flexi_rk_step_stages (storing
the five stage inputs of every step) and then applies flexi_adjoint_step to
each step of the segment in reverse order.  All arithmetic runs in the CUDA
kernels; torch provides the buffers.
"""
from __future__ import annotations

import torch


class RKAdjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, solver, nsteps: int, dt: float, t0: float = 0.0, checkpoint_every: int = 20):
        U = U0.detach().clone()
        dU = torch.zeros_like(U)
        ckpts = []
        for s in range(nsteps):
            if s % checkpoint_every == 0:
                ckpts.append(U.clone())
            solver.step(U, dU, t0 + s * dt, dt)
        ctx.solver, ctx.nsteps, ctx.dt, ctx.t0, ctx.C = solver, nsteps, dt, t0, checkpoint_every
        ctx.ckpts = ckpts
        return U

    @staticmethod
    def backward(ctx, gU):
        solver, nsteps, dt, t0, C = ctx.solver, ctx.nsteps, ctx.dt, ctx.t0, ctx.C
        lamU = gU.detach().clone().contiguous()
        lam_dU = torch.zeros_like(lamU)
        nseg = len(ctx.ckpts)
        stages = None
        for seg in reversed(range(nseg)):
            s0, s1 = seg * C, min(nsteps, (seg + 1) * C)
            if stages is None or stages.shape[0] < s1 - s0:
                stages = torch.empty((s1 - s0, 5) + tuple(lamU.shape), dtype=lamU.dtype, device=lamU.device)
            U = ctx.ckpts[seg].clone()
            dU = torch.zeros_like(U)
            for s in range(s0, s1):
                solver.step_stages(U, dU, t0 + s * dt, dt, stages[s - s0])
            for s in reversed(range(s0, s1)):
                solver.adjoint_step(stages[s - s0], lamU, lam_dU, t0 + s * dt, dt)
        ctx.ckpts = None
        return lamU, None, None, None, None, None


def final_state(U0, solver, nsteps, dt, t0=0.0, checkpoint_every=20):
    """U(T) = RK^nsteps(U0), differentiable with respect to U0 through the
    discrete adjoint."""
    return RKAdjoint.apply(U0, solver, nsteps, dt, t0, checkpoint_every)
