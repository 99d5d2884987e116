"""torch.autograd wrappers over the C ABI: the VJP of d u~/dt and RK4 rollouts with
checkpointing.  Marshalling only: forward and reverse passes run in libesd.so."""
import torch

from . import (esd_rhs, esd_rhs_save, esd_rhs_vjp, esd_rhs_vjp_saved, esd_rk_step, esd_rk_step_save,
               esd_rk_step_vjp, esd_rk_step_vjp_saved)


class Rhs(torch.autograd.Function):
    """d u~/dt = F(u~) with backward (dF/du~)^T g.

    save_tape=True (the default): the forward call keeps its entropy-projected states in a
    tape (esd_rhs_save, about 11 modal states of memory) and the backward reads them
    (esd_rhs_vjp_saved); False: nothing but u is kept and the backward recomputes the
    projection (esd_rhs_vjp).  Both give the same gradient bit for bit."""

    @staticmethod
    def forward(ctx, u, mesh, save_tape=True):
        u = u.contiguous()
        out = torch.empty_like(u)
        if save_tape:
            tape = mesh.empty_tapes()
            esd_rhs_save(mesh.handle, u, out, tape)
            ctx.save_for_backward(u, tape)
        else:
            esd_rhs(mesh.handle, u, out)
            ctx.save_for_backward(u)
        ctx.mesh = mesh
        return out

    @staticmethod
    def backward(ctx, g):
        saved = ctx.saved_tensors
        u = saved[0]
        grad = torch.empty_like(u)
        if len(saved) == 2:
            esd_rhs_vjp_saved(ctx.mesh.handle, u, saved[1], g.contiguous(), grad)
        else:
            esd_rhs_vjp(ctx.mesh.handle, u, g.contiguous(), grad)
        return grad, None, None


class RK4Rollout(torch.autograd.Function):
    """n_steps classical RK4 steps of size dt.

    checkpoint="stages": the four stage inputs of every step are stored during the forward
    pass (4 states per step) and the discrete adjoint runs directly on them, recomputing
    each stage's entropy projection;
    checkpoint="tapes": as "stages", plus each stage's forward tape (the entropy-projected
    states, about 11 modal states per stage), so that the adjoint does not recompute the
    projections;
    checkpoint="steps": only each step's input is stored and the stage inputs are recomputed
    step by step during the backward pass (1 state per step, one extra forward step each).
    """

    @staticmethod
    def forward(ctx, u0, mesh, dt, n_steps, checkpoint="stages"):
        u = u0.detach().clone().contiguous()
        tapes = None
        if checkpoint in ("stages", "tapes"):
            ck = torch.empty((n_steps, 4) + tuple(u.shape), dtype=u.dtype, device=u.device)
            # the step writes its stage inputs to one fixed buffer (so that its captured
            # CUDA graph is reused by every step) and they are copied into the checkpoint
            stage = torch.empty((4,) + tuple(u.shape), dtype=u.dtype, device=u.device)
            if checkpoint == "tapes":
                tapes = mesh.empty_tapes(n_steps, 4)
                tape = mesh.empty_tapes(4)
            for s in range(n_steps):
                if tapes is None:
                    esd_rk_step(mesh.handle, u, dt, stage)
                else:
                    esd_rk_step_save(mesh.handle, u, dt, stage, tape)
                    tapes[s].copy_(tape)
                ck[s].copy_(stage)
        elif checkpoint == "steps":
            ck = torch.empty((n_steps,) + tuple(u.shape), dtype=u.dtype, device=u.device)
            for s in range(n_steps):
                ck[s].copy_(u)
                esd_rk_step(mesh.handle, u, dt)
        else:
            raise ValueError(checkpoint)
        if tapes is None:
            ctx.save_for_backward(ck)
        else:
            ctx.save_for_backward(ck, tapes)
        ctx.mesh, ctx.dt, ctx.n, ctx.mode = mesh, dt, n_steps, checkpoint
        return u

    @staticmethod
    def backward(ctx, g):
        saved = ctx.saved_tensors
        ck = saved[0]
        mesh, dt = ctx.mesh, ctx.dt
        g = g.detach().clone().contiguous()
        if ctx.mode == "stages":
            for s in reversed(range(ctx.n)):
                esd_rk_step_vjp(mesh.handle, ck[s], dt, g, g)
        elif ctx.mode == "tapes":
            tapes = saved[1]
            for s in reversed(range(ctx.n)):
                esd_rk_step_vjp_saved(mesh.handle, ck[s], tapes[s], dt, g, g)
        else:
            stages = torch.empty((4,) + tuple(g.shape), dtype=g.dtype, device=g.device)
            tmp = torch.empty_like(g)
            for s in reversed(range(ctx.n)):
                tmp.copy_(ck[s])
                esd_rk_step(mesh.handle, tmp, dt, stages)
                esd_rk_step_vjp(mesh.handle, stages, dt, g, g)
        return g, None, None, None, None


def rollout(u0, mesh, dt, n_steps, checkpoint="stages"):
    return RK4Rollout.apply(u0, mesh, dt, n_steps, checkpoint)
