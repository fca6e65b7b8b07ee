"""torch.autograd.Function over the IMEX trajectory map (argument marshalling only).

``trajectory(problem, x0, obs_steps, ckpt_slots)`` returns the states X_n at the
requested steps (stacked along a new leading axis).  Its backward pass is one call of
``spadj_vjp``: the discrete adjoint sweep of the timestepper (Supplementary A.4) with the
incoming cotangents injected at the observation steps, recomputing the forward segments
from binomial checkpoints (RK problems) so long horizons fit in device memory.  Complex
tensors follow torch's convention for real losses, grad = dL/dRe + i dL/dIm, which is the
gradient for the real inner product the library's adjoints are defined with.
"""
import torch


class Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, problem, obs_steps, ckpt_slots):
        x0 = x0.detach().contiguous()
        n_steps = max(obs_steps)
        if n_steps < 1:
            raise ValueError("obs_steps must contain a step >= 1")
        if len(obs_steps) == 1:
            out = torch.empty_like(x0)
            problem.forward(n_steps, x0, out)
            outs = out.unsqueeze(0)
        else:
            traj = torch.empty((n_steps + 1,) + tuple(x0.shape), dtype=x0.dtype, device=x0.device)
            problem.forward(n_steps, x0, traj[-1], traj)
            outs = traj[list(obs_steps)].contiguous()
        ctx.save_for_backward(x0)
        ctx.problem, ctx.obs_steps, ctx.n_steps, ctx.ckpt = problem, tuple(obs_steps), n_steps, ckpt_slots
        return outs

    @staticmethod
    def backward(ctx, gout):
        (x0,) = ctx.saved_tensors
        g = torch.empty_like(x0)
        ctx.problem.vjp(x0, ctx.n_steps, ctx.obs_steps, gout.contiguous(), g, ckpt_slots=ctx.ckpt)
        return g, None, None, None


def trajectory(problem, x0, obs_steps, ckpt_slots=0):
    """States at `obs_steps` (tuple of ints), differentiable with respect to x0."""
    steps = tuple(int(s) for s in obs_steps)
    if len(set(steps)) != len(steps):
        raise ValueError("obs_steps must be distinct")
    return Trajectory.apply(x0, problem, steps, ckpt_slots)
