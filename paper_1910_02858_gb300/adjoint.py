"""Checkpointed discrete adjoint of the LSERK4(5) time integration as a
torch.autograd.Function.

forward(U0) runs nsteps RK steps.  It keeps U at the start of every
`checkpoint_every`-th step (dU need not be kept: A_1 = 0 makes the first stage
overwrite it), and for the last segment it stores the five stage inputs of
every step directly (flexi_rk_step_stages), so that segment is never
recomputed.  backward(gU_T) walks the segments in reverse: it recomputes each
earlier segment from its checkpoint with flexi_rk_step_stages and applies
flexi_adjoint_step to each step of the segment in reverse order.  All
arithmetic runs in the CUDA kernels; torch provides the buffers.
"""
from __future__ import annotations

import torch


class RKAdjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, solver, nsteps: int, dt: float, t0: float = 0.0, checkpoint_every: int = 20):
        C = checkpoint_every
        U = U0.detach().clone()
        dU = torch.zeros_like(U)
        nseg = (nsteps + C - 1) // C
        last0 = (nseg - 1) * C
        ckpts = []
        # room for one full segment (the last one may be shorter)
        stages = torch.empty((min(C, nsteps), 5) + tuple(U.shape), dtype=U.dtype, device=U.device)
        for s in range(nsteps):
            if s % C == 0 and s < last0:
                ckpts.append(U.clone())
            if s >= last0:
                solver.step_stages(U, dU, t0 + s * dt, dt, stages[s - last0])
            else:
                solver.step(U, dU, t0 + s * dt, dt)
        ctx.solver, ctx.nsteps, ctx.dt, ctx.t0, ctx.C = solver, nsteps, dt, t0, C
        ctx.ckpts, ctx.stages = ckpts, stages
        return U

    @staticmethod
    def backward(ctx, gU):
        solver, nsteps, dt, t0, C = ctx.solver, ctx.nsteps, ctx.dt, ctx.t0, ctx.C
        lamU = gU.detach().clone().contiguous()
        lam_dU = torch.zeros_like(lamU)
        nseg = (nsteps + C - 1) // C
        stages = ctx.stages
        for seg in reversed(range(nseg)):
            s0, s1 = seg * C, min(nsteps, (seg + 1) * C)
            if seg < nseg - 1:  # recompute the stage inputs of this segment from its checkpoint
                U = ctx.ckpts[seg].clone()
                dU = torch.zeros_like(U)
                for s in range(s0, s1):
                    solver.step_stages(U, dU, t0 + s * dt, dt, stages[s - s0])
            for s in reversed(range(s0, s1)):
                solver.adjoint_step(stages[s - s0], lamU, lam_dU, t0 + s * dt, dt)
        ctx.ckpts, ctx.stages = None, None
        return lamU, None, None, None, None, None


def final_state(U0, solver, nsteps, dt, t0=0.0, checkpoint_every=20):
    """U(T) = RK^nsteps(U0), differentiable with respect to U0 through the
    discrete adjoint."""
    return RKAdjoint.apply(U0, solver, nsteps, dt, t0, checkpoint_every)
