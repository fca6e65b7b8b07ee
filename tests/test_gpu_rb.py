"""GPU parity for the Rayleigh-Benard path (Fourier x Chebyshev-tau, RK222) through the
C-ABI against the FP64 oracle: transforms and their adjoints, the explicit term with its
JVP/VJP, the pencil solve and its adjoint, forward/tangent/adjoint trajectories, the
checkpointed gradient, and properties of the full configuration (256 x 64, Ra = 1e6,
dt = 1e-3, 2000 steps, binomial checkpointing)."""
import numpy as np
import pytest

import synthetic
from oracle import imex
from oracle import rayleigh_benard as orb
from tests.gpu_util import TOL, dev, host, rel_err
from tests.rb_util import F_T, F_T_jvp, F_T_vjp, gpu_problem, stage_solve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = [(16, 12), (32, 16), (256, 64)]


def _rand_state(o, seed, amp=1.0):
    s = synthetic.random_coeffs((3, o.Kx, o.N), seed=seed, scale=amp)
    s[:, 0] = s[:, 0].real
    return s


def _z(shape):
    return torch.zeros(shape, dtype=torch.complex128, device="cuda")


@pytest.mark.parametrize("Nx,Nz", SMALL)
def test_transforms(Nx, Nz):
    from paper_2506_14792_gb300 import spadj
    o = orb.RayleighBenard(Nx, Nz, 1e6)
    p = gpu_problem(Nx, Nz)
    c = synthetic.random_coeffs((o.Kx, o.N), seed=Nx)
    c[0] = c[0].real
    g = np.random.default_rng(Nz).standard_normal((o.Mz, o.Mx))
    og = torch.zeros((o.Mz, o.Mx), dtype=torch.float64, device="cuda")
    oc = _z((o.Kx, o.N))
    p.transform(spadj.C2G, dev(c), og)
    assert rel_err(host(og), o.c2g(c)) < 1e-13
    p.transform(spadj.G2C_ADJ, dev(c), og)
    assert rel_err(host(og), o.g2c_adj(c)) < 1e-13
    p.transform(spadj.G2C, dev(g), oc)
    assert rel_err(host(oc), o.g2c(g)) < 1e-13
    p.transform(spadj.C2G_ADJ, dev(g), oc)
    assert rel_err(host(oc), o.c2g_adj(g)) < 1e-13


@pytest.mark.parametrize("Nx,Nz", SMALL)
def test_F_jvp_vjp(Nx, Nz):
    o = orb.RayleighBenard(Nx, Nz, 1e6)
    p = gpu_problem(Nx, Nz)
    s = _rand_state(o, 1)
    d = _rand_state(o, 2)
    X = o.pencils(s)
    out = _z((3, o.Kx, o.N))
    p.eval_F(dev(s), out)
    assert rel_err(host(out), F_T(o, X)) < 1e-12
    p.eval_F_jvp(dev(s), dev(d), out)
    assert rel_err(host(out), F_T_jvp(o, X, o.pencils(d))) < 1e-12
    p.eval_F_vjp(dev(s), dev(d), out)
    assert rel_err(host(out), F_T_vjp(o, X, d)) < 1e-12


@pytest.mark.parametrize("Nx,Nz", SMALL)
def test_pencil_solve_and_adjoint(Nx, Nz):
    dt = 1e-3
    o = orb.RayleighBenard(Nx, Nz, 1e6)
    p = gpu_problem(Nx, Nz, dt=dt)
    v = _rand_state(o, 3)
    out = _z((3, o.Kx, o.N))
    b = dt * imex.RK222_GAMMA
    p.solve(dev(v), out)
    assert rel_err(host(out), stage_solve(o, v, b)) < 1e-12
    p.solve(dev(v), out, transpose=True)
    assert rel_err(host(out), stage_solve(o, v, b, transpose=True)) < 1e-12


@pytest.fixture(scope="module")
def small_case():
    Nx, Nz, dt, nsteps = 16, 12, 1e-2, 30
    o = orb.RayleighBenard(Nx, Nz, 1e6)
    s0 = synthetic.rb_ic(Nx, Nz, seed=2, amp=0.3)
    J, g, X, stages = orb.gradient(o, o.pencils(s0), nsteps, dt)
    return o, s0, J, g, X, stages, dt, nsteps


def test_largest_chebyshev_size_gradient():
    """Nz = 128 (the largest supported z resolution: the stage operators no longer fit the fused
    column kernel, so the separate kernels run) and a ragged Nx: gradient against the oracle."""
    Nx, Nz, dt, n = 24, 128, 2e-3, 3
    o = orb.RayleighBenard(Nx, Nz, 1e6)
    s0 = synthetic.rb_ic(Nx, Nz, seed=4, amp=0.3)
    J, g, X, stages = orb.gradient(o, o.pencils(s0), n, dt)
    p = gpu_problem(Nx, Nz, dt=dt)
    gr = _z((3, o.Kx, o.N))
    Jg = p.gradient(dev(s0), n, gr, ckpt_slots=2)
    assert abs(Jg[0] - J) <= TOL * abs(J)
    assert rel_err(host(gr), o.state(g)) < TOL


def test_forward_tangent_adjoint_trajectories(small_case):
    o, s0, J, g, X, stages, dt, nsteps = small_case
    p = gpu_problem(o.Nx, o.Nz, dt=dt)
    traj = _z((nsteps + 1, 3, o.Kx, o.N))
    xN = _z((3, o.Kx, o.N))
    p.forward(nsteps, dev(s0), xN, traj)
    assert rel_err(host(xN), o.state(X[-1])) < TOL
    assert rel_err(host(traj), np.stack([o.state(x) for x in X])) < TOL
    d0 = synthetic.rb_ic(o.Nx, o.Nz, seed=7, amp=1.0)
    dxN = _z((3, o.Kx, o.N))
    p.tangent(nsteps, dev(s0), dev(d0), dxN)
    A, H = imex.rk222_tableaux()
    dX = imex.rk_tangent(o, stages, o.pencils(d0), dt, A, H)
    assert rel_err(host(dxN), o.state(dX[-1])) < TOL
    yN = o.state(o.kinetic_energy_grad(X[-1]))
    gr = _z((3, o.Kx, o.N))
    p.adjoint(nsteps, traj, dev(yN), gr)
    assert rel_err(host(gr), o.state(g)) < TOL


@pytest.mark.parametrize("Nx,Nz,nonlinear", [(16, 12, True), (32, 16, True), (16, 12, False)])
def test_rk443_forward_tangent_adjoint_gradient(Nx, Nz, nonlinear):
    """ARS(4,4,3) on the separate kernels: trajectory, tangent, adjoint over the stored trajectory
    and the checkpointed gradient against the oracle's RK stage equation and its adjoint."""
    from paper_2506_14792_gb300 import spadj
    dt, nsteps = 1e-2, 10
    o = orb.RayleighBenard(Nx, Nz, 1e6, nonlinear=nonlinear)
    s0 = synthetic.rb_ic(Nx, Nz, seed=2, amp=0.3)
    tab = imex.rk443_tableaux()
    J, g, X, stages = orb.gradient(o, o.pencils(s0), nsteps, dt, tab)
    p = gpu_problem(Nx, Nz, dt=dt, scheme=spadj.SPADJ_RK443, nonlinear=nonlinear)
    traj = _z((nsteps + 1, 3, o.Kx, o.N))
    xN = _z((3, o.Kx, o.N))
    p.forward(nsteps, dev(s0), xN, traj)
    assert rel_err(host(traj), np.stack([o.state(x) for x in X])) < TOL
    d0 = synthetic.rb_ic(Nx, Nz, seed=7, amp=1.0)
    dxN = _z((3, o.Kx, o.N))
    p.tangent(nsteps, dev(s0), dev(d0), dxN)
    dX = imex.rk_tangent(o, stages, o.pencils(d0), dt, *tab)
    assert rel_err(host(dxN), o.state(dX[-1])) < TOL
    yN = o.state(o.kinetic_energy_grad(X[-1]))
    gr = _z((3, o.Kx, o.N))
    p.adjoint(nsteps, traj, dev(yN), gr)
    assert rel_err(host(gr), o.state(g)) < TOL
    gc = _z((3, o.Kx, o.N))
    Jg = p.gradient(dev(s0), nsteps, gc, ckpt_slots=3)
    assert abs(Jg[0] - J) <= TOL * abs(J)
    assert rel_err(host(gc), o.state(g)) < TOL


@pytest.mark.parametrize("scheme", ["rk222", "rk443"])
def test_step_size_schedule(scheme):
    """Step-dependent sizes (a stage factorisation per distinct size): trajectory, adjoint over
    it and the checkpointed two-lane gradient against the oracle under the same schedule; an
    empty schedule restores the constant step."""
    from paper_2506_14792_gb300 import spadj
    Nx, Nz = 16, 12
    sched = [1e-2, 1e-2, 4e-3, 4e-3, 4e-3, 7e-3, 1e-2, 2e-3, 7e-3, 1e-2]
    n = len(sched)
    o = orb.RayleighBenard(Nx, Nz, 1e6)
    s0 = synthetic.rb_ic(Nx, Nz, seed=2, amp=0.3)
    tab = imex.rk222_tableaux() if scheme == "rk222" else imex.rk443_tableaux()
    sch = spadj.SPADJ_RK222 if scheme == "rk222" else spadj.SPADJ_RK443
    J, g, X, stages = orb.gradient(o, o.pencils(s0), n, sched, tab)
    p = gpu_problem(Nx, Nz, dt=1e-2, scheme=sch)
    p.set_dt_schedule(sched)
    traj = _z((n + 1, 3, o.Kx, o.N))
    xN = _z((3, o.Kx, o.N))
    p.forward(n, dev(s0), xN, traj)
    assert rel_err(host(traj), np.stack([o.state(x) for x in X])) < TOL
    yN = o.state(o.kinetic_energy_grad(X[-1]))
    gr = _z((3, o.Kx, o.N))
    p.adjoint(n, traj, dev(yN), gr)
    assert rel_err(host(gr), o.state(g)) < TOL
    gc = _z((3, o.Kx, o.N))
    Jg = p.gradient(dev(s0), n, gc, ckpt_slots=3)
    assert abs(Jg[0] - J) <= TOL * abs(J)
    assert rel_err(host(gc), o.state(g)) < TOL
    with pytest.raises(spadj.SpadjError):
        p.gradient(dev(s0), n + 1, gc)  # longer than the schedule
    p.set_dt_schedule([])
    g1 = _z((3, o.Kx, o.N))
    p.gradient(dev(s0), 6, g1, ckpt_slots=3)
    q = gpu_problem(Nx, Nz, dt=1e-2, scheme=sch)
    g2 = _z((3, o.Kx, o.N))
    q.gradient(dev(s0), 6, g2, ckpt_slots=3)
    assert torch.equal(g1, g2)


@pytest.mark.parametrize("slots", [0, 2, 5, 31])
def test_checkpointed_gradient(small_case, slots):
    o, s0, J, g, X, stages, dt, nsteps = small_case
    p = gpu_problem(o.Nx, o.Nz, dt=dt)
    gr = _z((3, o.Kx, o.N))
    Jg = p.gradient(dev(s0), nsteps, gr, ckpt_slots=slots)
    assert abs(Jg[0] - J) <= TOL * abs(J)
    assert rel_err(host(gr), o.state(g)) < TOL
    ref = _z((3, o.Kx, o.N))
    p.gradient(dev(s0), nsteps, ref, ckpt_slots=0)
    assert torch.equal(gr, ref)  # recomputation is bitwise identical to store-all


@pytest.mark.parametrize("slots,hslots", [(2, 3), (1, 5), (4, 2), (3, 40)])
def test_two_level_checkpointing(small_case, slots, hslots):
    """Device slots plus host slots (the two-level schedule): gradient and a seeded VJP equal
    the store-all sweep bitwise."""
    o, s0, J, g, X, stages, dt, nsteps = small_case
    p = gpu_problem(o.Nx, o.Nz, dt=dt)
    ref = _z((3, o.Kx, o.N))
    Jr = p.gradient(dev(s0), nsteps, ref, ckpt_slots=0)
    p.set_option(9, hslots)
    gr = _z((3, o.Kx, o.N))
    Jg = p.gradient(dev(s0), nsteps, gr, ckpt_slots=slots)
    assert Jg[0] == Jr[0] and torch.equal(gr, ref)
    steps = [0, nsteps // 2, nsteps]
    seeds = dev(np.stack([_rand_state(o, 50 + i) for i in range(3)]))
    v_host = _z((3, o.Kx, o.N))
    p.vjp(dev(s0), nsteps, steps, seeds, v_host, ckpt_slots=slots)
    p.set_option(9, 0)
    v_ref = _z((3, o.Kx, o.N))
    p.vjp(dev(s0), nsteps, steps, seeds, v_ref, ckpt_slots=0)
    assert torch.equal(v_host, v_ref)


def test_gpu_dot_test(small_case):
    o, s0, J, g, X, stages, dt, nsteps = small_case
    p = gpu_problem(o.Nx, o.Nz, dt=dt)
    traj = _z((nsteps + 1, 3, o.Kx, o.N))
    xN = _z((3, o.Kx, o.N))
    p.forward(nsteps, dev(s0), xN, traj)
    for seed in range(3):
        d0 = synthetic.rb_ic(o.Nx, o.Nz, seed=20 + seed, amp=1.0)
        yN = _rand_state(o, 40 + seed)
        dxN = _z((3, o.Kx, o.N))
        p.tangent(nsteps, dev(s0), dev(d0), dxN)
        gr = _z((3, o.Kx, o.N))
        p.adjoint(nsteps, traj, dev(yN), gr)
        lhs = imex.inner(host(gr), d0)
        rhs = imex.inner(yN, host(dxN))
        assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_linear_problem_matches_oracle():
    Nx, Nz, dt, nsteps = 16, 16, 5e-3, 40
    o = orb.RayleighBenard(Nx, Nz, 2e3, nonlinear=False)
    p = gpu_problem(Nx, Nz, Ra=2e3, dt=dt, nonlinear=False)
    s0 = synthetic.rb_ic(Nx, Nz, seed=3, amp=1.0)
    A, H = imex.rk222_tableaux()
    X, _ = imex.rk_forward(o, o.pencils(s0), nsteps, dt, A, H)
    xN = _z((3, o.Kx, o.N))
    p.forward(nsteps, dev(s0), xN)
    assert rel_err(host(xN), o.state(X[-1])) < TOL


def test_full_size_short_horizon_vs_oracle():
    """256 x 64, Ra = 1e6, dt = 1e-3: 12 steps of the full configuration against the oracle."""
    Nx, Nz, dt, nsteps = 256, 64, 1e-3, 12
    o = orb.RayleighBenard(Nx, Nz, 1e6)
    s0 = synthetic.rb_ic(Nx, Nz, seed=2, amp=1e-3)
    J, g, X, _ = orb.gradient(o, o.pencils(s0), nsteps, dt)
    p = gpu_problem(Nx, Nz, dt=dt)
    gr = _z((3, o.Kx, o.N))
    Jg = p.gradient(dev(s0), nsteps, gr, ckpt_slots=4)
    assert abs(Jg[0] - J) <= TOL * abs(J)
    assert rel_err(host(gr), o.state(g)) < TOL


def test_full_config_properties():
    """Full configuration (2000 steps, 64 slots): checkpointed gradient equals the store-all
    gradient bitwise, and matches central finite differences of the GPU forward map."""
    Nx, Nz, dt, nsteps = 256, 64, 1e-3, 2000
    p = gpu_problem(Nx, Nz, dt=dt)
    s0 = synthetic.rb_ic(Nx, Nz, seed=2, amp=1e-3)
    gr = _z((3, Nx // 2, Nz))
    J = p.gradient(dev(s0), nsteps, gr, ckpt_slots=64)[0]
    ref = _z((3, Nx // 2, Nz))
    p.gradient(dev(s0), nsteps, ref, ckpt_slots=0)
    assert torch.equal(gr, ref)
    assert np.isfinite(J) and J > 0
    gh = host(gr)
    xN = _z((3, Nx // 2, Nz))
    Jd = torch.zeros(1, dtype=torch.float64, device="cuda")
    seed = _z((3, Nx // 2, Nz))
    def Jof(s):
        p.forward(nsteps, dev(s), xN)
        p.objective(xN, Jd, seed)
        return float(Jd.item())
    assert abs(Jof(s0) - J) <= 1e-13 * abs(J)
    for k in range(2):
        d = synthetic.rb_ic(Nx, Nz, seed=60 + k, amp=1.0)
        eps = 1e-4 * np.linalg.norm(s0) / np.linalg.norm(d)
        fd = (Jof(s0 + eps * d) - Jof(s0 - eps * d)) / (2 * eps)
        assert abs(fd - imex.inner(gh, d)) <= 1e-6 * abs(fd)


def test_fused_column_stage_matches_separate_kernels():
    """The fused fold + solve + expand cluster kernel and the three separate kernels compute the
    same gradient (the summation order of the fold differs, so agreement is to rounding)."""
    Nx, Nz, n = 32, 16, 8
    o = orb.RayleighBenard(Nx, Nz, 1e6)
    s0 = synthetic.rb_ic(Nx, Nz, seed=2, amp=0.3)
    out = []
    for fuse in (1, 0):
        p = gpu_problem(Nx, Nz, dt=1e-2)
        p.set_option(7, fuse)
        g = _z((3, o.Kx, o.N))
        J = p.gradient(dev(s0), n, g, ckpt_slots=3)
        out.append((J[0], host(g)))
    assert abs(out[0][0] - out[1][0]) <= 1e-13 * abs(out[1][0])
    assert rel_err(out[0][1], out[1][1]) < 1e-12


@pytest.mark.parametrize("Nx,Nz", [(16, 12), (256, 64)])
def test_x_rows_per_cta_bitwise(Nx, Nz):
    """The multi-row x FFT (rows interleaved, transformed together) performs the same
    arithmetic per row as the one-row kernel: F and its VJP agree bitwise for 1, 2, 4 rows."""
    o = orb.RayleighBenard(Nx, Nz, 1e6)
    s, d = _rand_state(o, 7), _rand_state(o, 8)
    outs = []
    for nb in (1, 2, 4):
        p = gpu_problem(Nx, Nz)
        p.set_option(8, nb)
        f = _z((3, o.Kx, o.N))
        v = _z((3, o.Kx, o.N))
        p.eval_F(dev(s), f)
        p.eval_F_vjp(dev(s), dev(d), v)
        outs.append((f, v))
    for f, v in outs[1:]:
        assert torch.equal(f, outs[0][0]) and torch.equal(v, outs[0][1])


def test_full_horizon_gradient_matches_oracle_golden():
    """The benchmarked configuration itself (256 x 64, Ra = 1e6, RK222, dt = 1e-3, 2000 steps, 64
    binomial checkpoint slots): J and dJ/dX_0 against the oracle's values in tests/golden (written by
    tests/golden/make_rb_256x64_2000steps.py from oracle/ alone), element by element.  The bar is
    max(1e-10, 10 x the oracle's own spread), the spread being the difference between the oracle run
    with numpy's FFT and with direct exponential sums (about 1e-14 at this horizon)."""
    import os
    gold = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                "rb_256x64_ra1e6_rk222_2000steps.npz"))
    tol = max(1e-10, 10.0 * float(gold["spread_grad"]), 10.0 * float(gold["spread_J"]))
    assert tol == 1e-10  # the spread is far below the parity bar at this horizon
    Nx, Nz, dt, nsteps = 256, 64, 1e-3, 2000
    p = gpu_problem(Nx, Nz, dt=dt)
    s0 = synthetic.rb_ic(Nx, Nz, seed=2, amp=1e-3)
    gr = _z((3, Nx // 2, Nz))
    J = p.gradient(dev(s0), nsteps, gr, ckpt_slots=64)[0]
    assert abs(J - float(gold["J"])) <= tol * abs(float(gold["J"]))
    assert rel_err(host(gr), gold["grad"]) < tol
