"""torch.autograd wrappers over the C ABI: the VJP of d u~/dt and RK4 rollouts with
checkpointing.  Marshalling only: forward and reverse passes run in libesd.so."""
import torch

from . import esd_rhs, esd_rhs_vjp, esd_rk_step, esd_rk_step_vjp


class Rhs(torch.autograd.Function):
    """d u~/dt = F(u~) with backward (dF/du~)^T g (esd_rhs_vjp)."""

    @staticmethod
    def forward(ctx, u, mesh):
        u = u.contiguous()
        out = torch.empty_like(u)
        esd_rhs(mesh.handle, u, out)
        ctx.save_for_backward(u)
        ctx.mesh = mesh
        return out

    @staticmethod
    def backward(ctx, g):
        (u,) = ctx.saved_tensors
        grad = torch.empty_like(u)
        esd_rhs_vjp(ctx.mesh.handle, u, g.contiguous(), grad)
        return grad, None


class RK4Rollout(torch.autograd.Function):
    """n_steps classical RK4 steps of size dt.

    checkpoint="stages": the four stage inputs of every step are stored during the forward
    pass (4 states per step) and the discrete adjoint runs directly on them;
    checkpoint="steps": only each step's input is stored and the stage inputs are recomputed
    step by step during the backward pass (1 state per step, one extra forward step each).
    """

    @staticmethod
    def forward(ctx, u0, mesh, dt, n_steps, checkpoint="stages"):
        u = u0.detach().clone().contiguous()
        if checkpoint == "stages":
            ck = torch.empty((n_steps, 4) + tuple(u.shape), dtype=u.dtype, device=u.device)
            # the step writes its stage inputs to one fixed buffer (so that its captured
            # CUDA graph is reused by every step) and they are copied into the checkpoint
            stage = torch.empty((4,) + tuple(u.shape), dtype=u.dtype, device=u.device)
            for s in range(n_steps):
                esd_rk_step(mesh.handle, u, dt, stage)
                ck[s].copy_(stage)
        elif checkpoint == "steps":
            ck = torch.empty((n_steps,) + tuple(u.shape), dtype=u.dtype, device=u.device)
            for s in range(n_steps):
                ck[s].copy_(u)
                esd_rk_step(mesh.handle, u, dt)
        else:
            raise ValueError(checkpoint)
        ctx.save_for_backward(ck)
        ctx.mesh, ctx.dt, ctx.n, ctx.mode = mesh, dt, n_steps, checkpoint
        return u

    @staticmethod
    def backward(ctx, g):
        (ck,) = ctx.saved_tensors
        mesh, dt = ctx.mesh, ctx.dt
        g = g.detach().clone().contiguous()
        if ctx.mode == "stages":
            for s in reversed(range(ctx.n)):
                esd_rk_step_vjp(mesh.handle, ck[s], dt, g, g)
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
