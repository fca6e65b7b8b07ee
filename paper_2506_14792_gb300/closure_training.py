"""Training of the learned closure through the coarse adjoint (argument marshalling and the
training loop only; every solve, transform, CNN pass, gradient, restriction and optimiser
update runs in libspadj.so).

Fine trajectories come from the library's own Kolmogorov solver at the fine resolution;
the training loss over an unrolled window of coarse steps is the 4D-Var misfit
sum_m 1/2 ||R(w_fine(t_m)) - w_coarse(t_m; p)||^2, R the spectral truncation to the coarse
grid, and its gradient with respect to the CNN parameters p comes from spadj_gradient's
adjoint sweep (eq. 6 with p entering F).  Adam (spadj_adam) updates p.
"""
import numpy as np
import torch

from . import spadj


def restrict(fine, nmem, Nf, Nc):
    """fine [..., nmem * Nf/2 * Nf] (complex, device) -> [..., nmem * Nc/2 * Nc]: the spectral
    truncation R of every member (spadj_restrict)."""
    lead = fine.shape[:-1]
    f = fine.reshape(-1, nmem * (Nf // 2) * Nf)
    out = torch.empty((f.shape[0], nmem * (Nc // 2) * Nc), dtype=fine.dtype, device=fine.device)
    p = spadj.Problem(spadj.SPADJ_KOLMOGOROV2D, spadj.SPADJ_SBDF2, [Nc], [2 * np.pi], [1.0, 0.0], 1.0, batch=nmem)
    for i in range(f.shape[0]):
        p.restrict(Nf, f[i], out[i])
    p.close()
    return out.reshape(lead + (nmem * (Nc // 2) * Nc,))


def spin_up(x0_fine, nmem, Nf, Re, dt_f, nsteps):
    """Advance fine initial states nsteps fine steps (so the training windows start from
    developed flow rather than from the synthetic spectra)."""
    p = spadj.Problem(spadj.SPADJ_KOLMOGOROV2D, spadj.SPADJ_SBDF2, [Nf], [2 * np.pi], [Re, 0.0], dt_f, batch=nmem)
    y = torch.empty_like(x0_fine)
    p.forward(nsteps, x0_fine, y)
    p.close()
    return y


def make_dataset(x0_fine, nmem, Nf, Nc, Re, dt_f, ratio, ncoarse, spin=0, chunk=64):
    """Restricted fine snapshots [ncoarse + 1][nmem * Nc/2 * Nc] for fine initial states
    x0_fine (concatenated members), generated `chunk` members at a time by the library's own
    fine solver (spun up `spin` fine steps first)."""
    per = (Nf // 2) * Nf
    out = []
    for c in range(0, nmem, chunk):
        k = min(chunk, nmem - c)
        x = x0_fine[c * per:(c + k) * per].contiguous()
        if spin:
            x = spin_up(x, k, Nf, Re, dt_f, spin)
        f = fine_snapshots(x, k, Nf, Re, dt_f, ratio, ncoarse)
        out.append(restrict(f, k, Nf, Nc))
        del f
    return torch.cat(out, dim=1).contiguous()


def train_selected(params, train_snaps, ntrain, val_snaps, nval, Nc, Re, dt_c, iters, every=25, lr=3e-3,
                   log=None):
    """Adam on the training windows with model selection on held-aside validation windows:
    every `every` iterations the summed validation error at T/4, T/2 and T is evaluated and the
    best parameters so far are kept (early stopping).  Returns (best params, history)."""
    nco = train_snaps.shape[0] - 1
    at = [nco // 4, nco // 2, nco]
    best, best_p, hist = None, params.clone(), []
    done = 0
    while done < iters:
        train(params, train_snaps, ntrain, Nc, Re, dt_c, every, lr=lr)
        done += every
        v = rollout_errors(params, val_snaps, nval, Nc, Re, dt_c, at)
        score = float(sum(v[k].mean() for k in at))
        hist.append((done, score))
        if log is not None:
            log(done, score)
        if best is None or score < best:
            best, best_p = score, params.clone()
    return best_p, hist


def fine_snapshots(x0_fine, nmem, Nf, Re, dt_f, ratio, ncoarse):
    """Fine trajectories from the library's solver; states every `ratio` fine steps."""
    p = spadj.Problem(spadj.SPADJ_KOLMOGOROV2D, spadj.SPADJ_SBDF2, [Nf], [2 * np.pi], [Re, 0.0], dt_f, batch=nmem)
    nf = ratio * ncoarse
    traj = torch.empty((nf + 1,) + tuple(x0_fine.shape), dtype=x0_fine.dtype, device=x0_fine.device)
    p.forward(nf, x0_fine, traj[-1], traj)
    snaps = traj[::ratio].clone()
    del traj
    p.close()
    return snaps  # [ncoarse + 1][state]


class Adam:
    """Adam moments of the closure parameters; the update itself runs in the library (spadj_adam)."""

    def __init__(self, problem, n, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, device="cuda"):
        self.p = problem
        self.m = torch.zeros(n, dtype=torch.float64, device=device)
        self.v = torch.zeros_like(self.m)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, params, g):
        self.t += 1
        self.p.adam(g, self.t, self.m, self.v, params, lr=self.lr, b1=self.b1, b2=self.b2, eps=self.eps)


def coarse_problem(nmem, Nc, Re, dt_c):
    return spadj.Problem(spadj.SPADJ_KOLMOGOROV2D, spadj.SPADJ_SBDF2, [Nc], [2 * np.pi], [Re, 0.0], dt_c, batch=nmem,
                         closure=True)


def train(params, coarse_snaps, nmem, Nc, Re, dt_c, iters, lr=1e-3, log=None):
    """Adam on the closure parameters; coarse_snaps [ncoarse + 1][state] (restricted fine states,
    the first one is the coarse initial condition).  Returns the per-iteration losses."""
    nco = coarse_snaps.shape[0] - 1
    p = coarse_problem(nmem, Nc, Re, dt_c)
    steps = list(range(1, nco + 1))
    p.set_observations(steps, coarse_snaps[1:].contiguous(), Nc // 2 - 1)
    opt = Adam(p, params.numel(), lr=lr, device=params.device)
    g = torch.empty_like(coarse_snaps[0])
    gp = torch.empty_like(params)
    losses = []
    for it in range(iters):
        p.set_params(params)
        J = p.gradient(coarse_snaps[0].contiguous(), nco, g, objective=spadj.SPADJ_OBJ_FOURDVAR, grad_p=gp)
        losses.append(float(np.sum(J)))
        opt.step(params, gp)
        if log is not None and it % 10 == 0:
            log(it, losses[-1])
    p.close()
    return losses


def rollout_errors(params, coarse_snaps, nmem, Nc, Re, dt_c, at_steps):
    """Relative coefficient-space errors ||w_c(t) - R(w_f(t))|| / ||R(w_f(t))|| per member at the
    given coarse steps, for the closure with `params` (zero parameters = plain coarse solver)."""
    nco = max(at_steps)
    p = coarse_problem(nmem, Nc, Re, dt_c)
    p.set_params(params)
    traj = torch.empty((nco + 1,) + tuple(coarse_snaps[0].shape), dtype=coarse_snaps.dtype, device=coarse_snaps.device)
    p.forward(nco, coarse_snaps[0].contiguous(), traj[-1], traj)
    out = {}
    K = (Nc // 2) * Nc
    for s in at_steps:
        d = (traj[s] - coarse_snaps[s]).reshape(nmem, K)
        r = coarse_snaps[s].reshape(nmem, K)
        out[s] = (d.abs().pow(2).sum(1).sqrt() / r.abs().pow(2).sum(1).sqrt()).cpu().numpy()
    p.close()
    return out
