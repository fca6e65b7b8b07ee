"""torch.autograd.Function over the IMEX trajectory map (argument marshalling only).

``trajectory(problem, x0, obs_steps, ckpt_slots)`` returns the states X_n at the
requested steps (stacked along a new leading axis).  Its backward pass is one call of
``spadj_vjp``: the discrete adjoint sweep of the timestepper (Supplementary A.4) with the
incoming cotangents injected at the observation steps, recomputing the forward segments
from binomial checkpoints so long horizons fit in device memory.  The forward pass keeps
only the requested states: one-step (Runge-Kutta) problems advance from one requested step
to the next with spadj_forward; multistep problems advance one step at a time on their
restart state (spadj_step_forward), since a new spadj_forward call would restart the scheme
at first order; problems without step entry points store the trajectory.  Complex tensors
follow torch's convention for real losses, grad = dL/dRe + i dL/dIm, which is the gradient
for the real inner product the library's adjoints are defined with.
"""
import torch


def _states_at(problem, x0, steps):
    """X_n for n in steps (ascending order not required), keeping O(1) extra states."""
    n_steps = max(steps)
    order = sorted(set(steps) - {0})
    got = {0: x0.clone()} if 0 in steps else {}
    rk = problem.state_len(5) == problem.state_len(0) and problem.state_len(4) == problem.state_len(0)
    if len(order) == 1 or rk:
        cur, n = x0, 0
        for m in order:
            nxt = torch.empty_like(x0)
            problem.forward(m - n, cur, nxt)
            got[m] = nxt
            cur, n = nxt, m
    elif problem.state_len(4) > 0:
        ns = problem.state_len(0)
        real = torch.view_as_real(x0) if x0.is_complex() else x0
        s = torch.zeros(problem.state_len(4), dtype=torch.float64, device=x0.device)
        s[:ns] = real.reshape(-1)
        t = torch.empty_like(s)
        for n in range(n_steps):
            problem.step_forward(n, s, t)
            s, t = t, s
            if n + 1 in got or (n + 1) not in order:
                continue
            xn = s[:ns].clone().view(real.shape)
            got[n + 1] = torch.view_as_complex(xn) if x0.is_complex() else xn
    else:
        traj = torch.empty((n_steps + 1,) + tuple(x0.shape), dtype=x0.dtype, device=x0.device)
        problem.forward(n_steps, x0, traj[-1], traj)
        for m in order:
            got[m] = traj[m]
    return torch.stack([got[m] for m in steps])


class Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, problem, obs_steps, ckpt_slots):
        x0 = x0.detach().contiguous()
        n_steps = max(obs_steps)
        if n_steps < 1 or min(obs_steps) < 0:
            raise ValueError("obs_steps must lie in 0..n with some step >= 1")
        outs = _states_at(problem, x0, obs_steps)
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
