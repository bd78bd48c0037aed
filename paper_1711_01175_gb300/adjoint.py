"""Receiver traces as a differentiable function of the medium.

`receiver_traces(material, solver, u0, dt, nsteps)` runs nsteps LSRK steps
from u0 with the per-element medium material = [rho, lam, mu] ([3, nel]
float64) and returns the velocity at the solver's receivers after each step,
[nsteps, nrec, 3].  Its backward pass is the hand-written discrete adjoint of
the library (dgw_adjoint_traces): the forward states are kept only every
`checkpoint_every` steps, and each segment's stage inputs are recomputed once
from its checkpoint inside the library, so device memory holds one segment of
stage inputs (5 states per step).  The gradient is exact for the
discrete scheme (agreement with finite differences of any misfit of the
traces up to their truncation error).
"""
from __future__ import annotations

import torch


class _ReceiverTraces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, material, solver, u0, dt, nsteps, checkpoint_every):
        m = material.detach().to("cpu", torch.float64).contiguous().numpy()
        solver.upload_material(m[0], m[1], m[2])
        u = u0.detach().clone()
        res = torch.zeros_like(u)
        traces = torch.empty((nsteps, solver.nrec, 3), dtype=torch.float64, device=u.device)
        checkpoints = {}
        for k in range(nsteps):
            if k % checkpoint_every == 0:
                checkpoints[k] = u.clone()
            solver.step(u, res, dt, 1, t0=k * dt)
            solver.sample_receivers(u, traces[k])
        ctx.solver, ctx.dt, ctx.nsteps, ctx.every = solver, dt, nsteps, checkpoint_every
        ctx.checkpoints = checkpoints
        ctx.material_device = material.device
        ctx.u_shape = u.shape
        return traces

    @staticmethod
    def backward(ctx, g_traces):
        solver, dt, nsteps, every = ctx.solver, ctx.dt, ctx.nsteps, ctx.every
        g = g_traces.contiguous()
        any_ckpt = next(iter(ctx.checkpoints.values()))
        lam_u = torch.zeros_like(any_ckpt)
        lam_r = torch.zeros_like(any_ckpt)
        grad = torch.zeros((3, solver.nel), dtype=torch.float64, device=any_ckpt.device)
        for s0 in sorted(ctx.checkpoints, reverse=True):
            s1 = min(s0 + every, nsteps)
            # one call per segment: the library recomputes the segment's stage
            # inputs from the checkpoint and injects the trace sources step by step
            solver.adjoint_traces(lam_u, lam_r, grad, ctx.checkpoints[s0], g[s0:s1].contiguous(), dt, s1 - s0,
                                  t0=s0 * dt)
        return grad.to(ctx.material_device), None, None, None, None, None


def receiver_traces(material, solver, u0, dt, nsteps, checkpoint_every=50):
    return _ReceiverTraces.apply(material, solver, u0, dt, nsteps, checkpoint_every)
