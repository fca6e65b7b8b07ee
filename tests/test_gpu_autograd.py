"""torch.autograd.Function over the trajectory map (binomial checkpointing behind
backward) against the FP64 oracle's adjoint recurrences."""
import numpy as np
import pytest

import synthetic
from oracle import burgers as obur
from oracle import imex
from oracle import rayleigh_benard as orb
from tests.gpu_util import TOL, dev, host, rel_err
from tests.rb_util import gpu_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("slots", [0, 3])
def test_rb_autograd_final_state_loss(slots):
    from paper_2506_14792_gb300.autograd import trajectory
    Nx, Nz, dt, nsteps = 16, 12, 1e-2, 25
    o = orb.RayleighBenard(Nx, Nz, 1e6)
    p = gpu_problem(Nx, Nz, dt=dt)
    s0 = synthetic.rb_ic(Nx, Nz, seed=2, amp=0.3)
    W = np.random.default_rng(1).random((3, o.Kx, o.N))
    v = synthetic.random_coeffs((3, o.Kx, o.N), seed=3)
    x0 = dev(s0).requires_grad_(True)
    XT = trajectory(p, x0, (nsteps,), ckpt_slots=slots)[0]
    loss = (dev(W) * XT.abs() ** 2).sum() + (dev(v).conj() * XT).real.sum()
    loss.backward()
    A, H = imex.rk222_tableaux()
    X, stages = imex.rk_forward(o, o.pencils(s0), nsteps, dt, A, H)
    seed = o.pencils(2 * W * o.state(X[-1]) + v)
    g = imex.rk_adjoint(o, stages, lambda n: seed if n == nsteps else None, dt, A, H)
    assert rel_err(host(x0.grad), o.state(g)) < TOL


def test_burgers_autograd_observation_misfit():
    """4D-Var-style misfit at intermediate steps: cotangents injected during the sweep."""
    from paper_2506_14792_gb300 import spadj
    from paper_2506_14792_gb300.autograd import trajectory
    N, B, dt = 64, 3, 1e-3
    obs = (10, 25, 40)
    p = spadj.Problem(spadj.SPADJ_BURGERS1D, spadj.SPADJ_SBDF2, [N], [2 * np.pi], [0.01], dt, batch=B)
    X0 = synthetic.burgers_ic(N, batch=B, seed=4)
    truth = synthetic.burgers_ic(N, batch=B, seed=5)
    o = obur.Burgers(N, 0.01)
    Xt = imex.multistep_forward(o, truth, max(obs), dt)
    ob = np.stack([Xt[n] for n in obs])
    x0 = dev(X0).requires_grad_(True)
    outs = trajectory(p, x0, obs)
    loss = 0.5 * ((outs - dev(ob)).abs() ** 2).sum()
    loss.backward()
    X = imex.multistep_forward(o, X0, max(obs), dt)
    dJ = lambda n: (X[n] - ob[obs.index(n)]) if n in obs else None
    g = imex.multistep_adjoint(o, X, dJ, dt)
    assert rel_err(host(x0.grad), g) < TOL
    lv = float(loss.detach())
    assert abs(lv - 0.5 * sum(np.sum(np.abs(X[n] - ob[i]) ** 2) for i, n in enumerate(obs))) < 1e-10 * lv


@pytest.mark.parametrize("scheme", [2, 4])
def test_autograd_forward_keeps_only_requested_states(scheme):
    """Several observation steps on a long multistep horizon: the forward pass advances the restart
    state one step at a time and stores only the observed states (no (n+1)-state trajectory), the
    gradient (checkpointed backward) equals the store-all one bitwise, and the states equal
    spadj_forward's."""
    from paper_2506_14792_gb300 import spadj
    from paper_2506_14792_gb300.autograd import trajectory
    N, B, dt, n = 256, 64, 1e-3, 400
    obs = (0, 50, 399, 400, 7)
    p = spadj.Problem(spadj.SPADJ_BURGERS1D, scheme, [N], [2 * np.pi], [0.01], dt, batch=B)
    X0 = dev(synthetic.burgers_ic(N, batch=B, seed=4))
    W = dev(synthetic.random_coeffs((len(obs), B, N // 2), seed=6))
    state_bytes = X0.numel() * 16
    grads = []
    for slots in (0, 6):
        x0 = X0.clone().requires_grad_(True)
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        outs = trajectory(p, x0, obs, ckpt_slots=slots)
        torch.cuda.synchronize()
        assert torch.cuda.max_memory_allocated() - base < 40 * state_bytes  # O(observations), not O(n) = 401
        for i, m in enumerate(obs):
            ref = torch.empty_like(X0)
            p.forward(m, X0, ref)
            assert torch.equal(outs[i], ref)
        (W.conj() * outs).real.sum().backward()
        grads.append(x0.grad)
    assert torch.equal(grads[0], grads[1])
