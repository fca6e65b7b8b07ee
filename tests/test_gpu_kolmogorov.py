"""GPU parity for the batched Kolmogorov path (mixed resolutions in one persistent launch,
SBDF2, 4D-Var) through the C-ABI against the FP64 oracle, plus the scheduler's failure path
(a bounded wait that runs out returns SPADJ_ERR_TIMEOUT and leaves the context usable)."""
import numpy as np
import pytest

import synthetic
from oracle import imex
from oracle import kolmogorov as okol
from tests.gpu_util import TOL, dev, host, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gpu_problem(sizes, Re=100.0, dt=5e-3, nonlinear=True, forcing=True):
    from paper_2506_14792_gb300 import spadj
    return spadj.Problem(spadj.SPADJ_KOLMOGOROV2D, spadj.SPADJ_SBDF2, [sizes[0]], [2 * np.pi], [Re, 0.0 if forcing else 1.0],
                         dt, batch=len(sizes), nonlinear=nonlinear, batch_n=list(sizes))


def pack(arrs):
    return np.concatenate([a.ravel() for a in arrs])


def unpack(v, sizes):
    out, o = [], 0
    for n in sizes:
        k = (n // 2) * n
        out.append(v[o:o + k].reshape(n // 2, n))
        o += k
    return out


def ics(sizes, seed0):
    return [okol.Kolmogorov(n, 100.0).project(synthetic.kolmogorov_ic(n, seed0 + i)) for i, n in enumerate(sizes)]


def test_eval_F_mixed():
    sizes = [16, 24, 32]
    p = gpu_problem(sizes)
    X = ics(sizes, 1)
    out = torch.zeros(sum((n // 2) * n for n in sizes), dtype=torch.complex128, device="cuda")
    p.eval_F(dev(pack(X)), out)
    got = unpack(host(out), sizes)
    for n, x, g in zip(sizes, X, got):
        assert rel_err(g, okol.Kolmogorov(n, 100.0).F(x)) < 1e-12


@pytest.mark.parametrize("persistent", [1, 0])
def test_forward_mixed_batch(persistent):
    sizes, dt, nsteps = [16, 24, 32, 16], 5e-3, 30
    p = gpu_problem(sizes, dt=dt)
    p.set_option(0, persistent)
    X = ics(sizes, 10)
    out = torch.zeros(sum((n // 2) * n for n in sizes), dtype=torch.complex128, device="cuda")
    p.forward(nsteps, dev(pack(X)), out)
    got = unpack(host(out), sizes)
    for n, x, g in zip(sizes, X, got):
        o = okol.Kolmogorov(n, 100.0)
        assert rel_err(g, imex.multistep_forward(o, x, nsteps, dt)[-1]) < TOL


def test_persistent_equals_phased_bitwise():
    sizes, nsteps = [16, 32, 48], 12
    X = dev(pack(ics(sizes, 20)))
    outs = []
    for mode in (1, 0):
        p = gpu_problem(sizes)
        p.set_option(0, mode)
        o = torch.zeros_like(X)
        p.forward(nsteps, X, o)
        outs.append(o)
    assert torch.equal(outs[0], outs[1])


def test_tilings_bitwise():
    """The tile sizes only group the same row and column transforms differently (x-modes per
    column tile, option 1; grid rows per row tile, option 2; resident CTAs per SM, option 3), so
    the forward states and the 4D-Var gradient are bitwise equal for every tiling, including tiles
    that do not divide the member (ragged last tiles)."""
    from paper_2506_14792_gb300 import spadj
    sizes, dt, nsteps, obs_steps, kmax = [16, 32, 48], 5e-3, 10, [5, 10], 6
    X0, obs, _, _ = _fourdvar_case(sizes, dt, nsteps, obs_steps, kmax, 40)
    X = dev(pack(X0))
    ref = None
    for cw, rw, cps in [(4, 2, 0), (2, 1, 0), (8, 4, 0), (3, 5, 0), (64, 64, 1), (1, 7, 2)]:
        p = gpu_problem(sizes, dt=dt)
        p.set_option(1, cw)
        p.set_option(2, rw)
        p.set_option(3, cps)
        p.set_observations(obs_steps, dev(obs), kmax)
        o = torch.zeros_like(X)
        p.forward(nsteps, X, o)
        g = torch.zeros_like(X)
        J = np.asarray(p.gradient(X, nsteps, g, objective=spadj.SPADJ_OBJ_FOURDVAR))
        if ref is None:
            ref = (o, g, J)
        else:
            assert torch.equal(o, ref[0]) and torch.equal(g, ref[1]) and np.array_equal(J, ref[2]), (cw, rw, cps)


def _fourdvar_case(sizes, dt, nsteps, obs_steps, kmax, seed0):
    X0 = ics(sizes, seed0)
    obs, Js, gs = [], [], []
    for i, n in enumerate(sizes):
        o = okol.Kolmogorov(n, 100.0)
        Xt = imex.multistep_forward(o, o.project(synthetic.kolmogorov_ic(n, 900 + seed0 + i)), nsteps, dt)
        mask = o.lowpass_mask(kmax)
        ob = np.stack([mask * Xt[k] for k in obs_steps])
        J, g, _ = okol.fourdvar_gradient(o, X0[i], nsteps, dt, obs_steps, ob, mask)
        obs.append(ob)
        Js.append(J)
        gs.append(g)
    obs_packed = np.stack([pack([obs[i][m] for i in range(len(sizes))]) for m in range(len(obs_steps))])
    return X0, obs_packed, Js, gs


@pytest.mark.parametrize("persistent", [1, 0])
def test_fourdvar_gradient_mixed(persistent):
    sizes, dt, nsteps, obs_steps, kmax = [16, 32, 48], 5e-3, 40, [10, 20, 30, 40], 8
    X0, obs, Js, gs = _fourdvar_case(sizes, dt, nsteps, obs_steps, kmax, 30)
    from paper_2506_14792_gb300 import spadj
    p = gpu_problem(sizes, dt=dt)
    p.set_option(0, persistent)
    p.set_observations(obs_steps, dev(obs), kmax)
    g = torch.zeros(sum((n // 2) * n for n in sizes), dtype=torch.complex128, device="cuda")
    J = p.gradient(dev(pack(X0)), nsteps, g, objective=spadj.SPADJ_OBJ_FOURDVAR)
    got = unpack(host(g), sizes)
    for i in range(len(sizes)):
        assert abs(J[i] - Js[i]) <= TOL * abs(Js[i])
        assert rel_err(got[i], gs[i]) < TOL


def test_vjp_final_seed():
    sizes, dt, nsteps = [16, 24], 5e-3, 25
    X0 = ics(sizes, 40)
    seeds = [synthetic.random_coeffs((n // 2, n), seed=70 + i) for i, n in enumerate(sizes)]
    p = gpu_problem(sizes, dt=dt)
    g = torch.zeros(sum((n // 2) * n for n in sizes), dtype=torch.complex128, device="cuda")
    p.vjp(dev(pack(X0)), nsteps, [nsteps], dev(pack(seeds)[None, :]), g)
    got = unpack(host(g), sizes)
    for i, n in enumerate(sizes):
        o = okol.Kolmogorov(n, 100.0)
        X = imex.multistep_forward(o, X0[i], nsteps, dt)
        want = imex.multistep_adjoint(o, X, lambda k: seeds[i] if k == nsteps else None, dt)
        assert rel_err(got[i], want) < TOL


def test_bounded_wait_times_out_and_context_survives():
    from paper_2506_14792_gb300 import spadj
    sizes = [16, 32]
    p = gpu_problem(sizes)
    X = dev(pack(ics(sizes, 50)))
    out = torch.zeros_like(X)
    p.set_option(4, 2000)   # short bounded wait
    p.set_option(5, 0)      # member 0's completions are never signalled
    with pytest.raises(spadj.SpadjError) as e:
        p.forward(5, X, out)
    assert e.value.status == spadj.SPADJ_ERR_TIMEOUT
    p.set_option(5, -1)
    p.set_option(4, 0)
    p.forward(5, X, out)  # the same problem and context still work
    torch.cuda.synchronize()
    o = okol.Kolmogorov(16, 100.0)
    got = unpack(host(out), sizes)
    x0 = unpack(host(X), sizes)
    assert rel_err(got[0], imex.multistep_forward(o, x0[0], 5, 5e-3)[-1]) < TOL


def test_autotune_keeps_results():
    sizes, nsteps = [16, 32], 10
    X = dev(pack(ics(sizes, 60)))
    p = gpu_problem(sizes)
    ref = torch.zeros_like(X)
    p.forward(nsteps, X, ref)
    p.autotune()
    out = torch.zeros_like(X)
    p.forward(nsteps, X, out)
    assert rel_err(host(out), host(ref)) < 1e-13


def test_full_batch_sampled_members():
    """64 members, 16 each at 128^2, 256^2, 384^2, 512^2, Re = 100, dt = 5e-4, one persistent
    launch per sweep; 4D-Var over a 40-step window (observations every 10 steps, |k| <= 32);
    one member per resolution checked against the oracle."""
    from paper_2506_14792_gb300 import spadj
    res = [128, 256, 384, 512]
    sizes = [res[i // 16] for i in range(64)]
    dt, nsteps, obs_steps, kmax = 5e-4, 40, [10, 20, 30, 40], 32
    X0 = [synthetic.kolmogorov_ic(n, 100 + i) for i, n in enumerate(sizes)]
    check = [0, 17, 34, 51]
    obs_m, ref = [], {}
    truth = {}
    for i in check:
        n = sizes[i]
        o = okol.Kolmogorov(n, 100.0)
        Xt = imex.multistep_forward(o, synthetic.kolmogorov_ic(n, 1000 + i), nsteps, dt)
        truth[i] = np.stack([o.lowpass_mask(kmax) * Xt[k] for k in obs_steps])
        J, g, _ = okol.fourdvar_gradient(o, X0[i], nsteps, dt, obs_steps, truth[i], o.lowpass_mask(kmax))
        ref[i] = (J, g)
    obs = np.stack([pack([truth[i][m] if i in truth else np.zeros((n // 2, n), complex)
                          for i, n in enumerate(sizes)]) for m in range(len(obs_steps))])
    p = gpu_problem(sizes, dt=dt)
    p.set_observations(obs_steps, dev(obs), kmax)
    g = torch.zeros(sum((n // 2) * n for n in sizes), dtype=torch.complex128, device="cuda")
    J = p.gradient(dev(pack(X0)), nsteps, g, objective=spadj.SPADJ_OBJ_FOURDVAR)
    got = unpack(host(g), sizes)
    assert np.all(np.isfinite(J))
    for i in check:
        assert abs(J[i] - ref[i][0]) <= TOL * abs(ref[i][0])
        assert rel_err(got[i], ref[i][1]) < TOL


@pytest.mark.parametrize("persistent", [1, 0])
def test_segmented_checkpointing_equals_store_all(persistent):
    """Checkpointed 4D-Var gradient: restart states [X_a, X_{a-1}, F(X_{a-1})] at segment starts (device
    slots, or page-locked host slots with option 9), each segment recomputed and reversed in one
    launch, the adjoint variables carried through the Y ring: bitwise equal to the store-all sweep,
    for J, dJ/dX_0 and spadj_vjp with cotangents injected at several steps."""
    from paper_2506_14792_gb300 import spadj
    sizes, dt, n = [16, 24, 32, 16], 5e-3, 40
    p = gpu_problem(sizes, dt=dt)
    p.set_option(0, persistent)
    X0 = dev(pack(ics(sizes, 30)))
    obs_steps = [7, 20, 33, 40]
    truth = dev(pack(ics(sizes, 70)))
    obs = torch.stack([truth * (0.5 + 0.1 * i) for i in range(len(obs_steps))]).contiguous()
    p.set_observations(obs_steps, obs, 5)
    ref = torch.zeros_like(X0)
    J = p.gradient(X0, n, ref, objective=spadj.SPADJ_OBJ_FOURDVAR, ckpt_slots=0)
    for slots, hs in ((3, 0), (5, 0), (39, 0), (0, 6)):
        p.set_option(9, hs)
        g = torch.zeros_like(X0)
        Jc = p.gradient(X0, n, g, objective=spadj.SPADJ_OBJ_FOURDVAR, ckpt_slots=slots)
        assert np.array_equal(Jc, J), (slots, hs)
        assert torch.equal(g, ref), (slots, hs)
    p.set_option(9, 0)
    seeds = torch.stack([dev(pack(ics(sizes, 90 + i))) for i in range(3)]).contiguous()
    ga, gb = torch.zeros_like(X0), torch.zeros_like(X0)
    p.vjp(X0, n, [n, 25, 3], seeds, ga, ckpt_slots=0)
    p.vjp(X0, n, [n, 25, 3], seeds, gb, ckpt_slots=4)
    assert torch.equal(ga, gb)


def test_step_entry_points_equal_sweeps():
    """spadj_step_forward on the restart state [X_n, X_{n-1}, F(X_{n-1})] reproduces spadj_forward, and
    the adjoint chain (seed step at N, then steps N-1..0 with cotangents injected as sources)
    reproduces spadj_vjp, bit for bit."""
    sizes, dt, n = [16, 24], 5e-3, 12
    p = gpu_problem(sizes, dt=dt)
    ns = p.state_len(0)
    assert p.state_len(4) == 3 * ns and p.state_len(5) == 2 * ns
    X0 = dev(pack(ics(sizes, 50)))
    s = torch.zeros(3 * ns, dtype=torch.float64, device="cuda")
    s[:ns] = torch.view_as_real(X0).reshape(-1)
    X = [s[:ns].clone()]
    for k in range(n):
        t = torch.zeros_like(s)
        p.step_forward(k, s, t)
        s = t
        X.append(s[:ns].clone())
    ref = torch.zeros_like(X0)
    p.forward(n, X0, ref)
    assert torch.equal(X[-1], torch.view_as_real(ref).reshape(-1))
    seeds = torch.stack([torch.view_as_real(dev(pack(ics(sizes, 60 + i)))).reshape(-1) for i in range(3)])
    at = {n: 0, 7: 1, 2: 2}
    y = None
    for k in range(n, -1, -1):
        out = torch.zeros(2 * ns, dtype=torch.float64, device="cuda")
        p.step_adjoint(k, X[k], y, out, src=seeds[at[k]].contiguous() if k in at else None)
        y = out
    g = torch.zeros_like(X0)
    p.vjp(X0, n, [n, 7, 2], torch.view_as_complex(seeds.reshape(3, -1, 2)).contiguous(), g)
    assert torch.equal(y[:ns], torch.view_as_real(g).reshape(-1))
