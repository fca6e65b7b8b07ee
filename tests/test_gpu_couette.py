"""GPU parity for the plane-Couette path (Fourier x, y x Chebyshev-tau z, SBDF1 -> SBDF2)
through the C-ABI against the FP64 oracle: transforms and their adjoints, the explicit term
u x omega with its JVP/VJP, the pencil step solve and its adjoint, forward/tangent/adjoint
trajectories, the energy-gain gradient with binomial checkpointing (checkpointed == store-all
bitwise), cotangent injection, and at the full size 128 x 64 x 64 (Re = 1000, dt = 5e-3)
the explicit term, sampled pencil solves and trajectory properties (dot test, central FD)."""
import numpy as np
import pytest

import synthetic
from oracle import couette as oco
from oracle import imex
from tests.gpu_util import TOL, dev, host, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = [(8, 4, 8), (16, 6, 12), (32, 8, 16)]
RE, DT = 1000.0, 5e-3


def gpu_problem(Nx, Ny, Nz, Re=RE, dt=DT, nonlinear=True, scheme=None, base="couette"):
    from paper_2506_14792_gb300 import spadj
    sch = spadj.SPADJ_SBDF2 if scheme is None else scheme
    b = {"couette": 0, "poiseuille": 1}[base]
    return spadj.Problem(spadj.SPADJ_COUETTE3D, sch, [Nx, Ny, Nz], [4 * np.pi, 2 * np.pi], [Re, b], dt,
                         nonlinear=nonlinear)


def to_gpu(s):
    """oracle fields (3, Kx, Ny, N) -> library layout (3, Ny, Kx, N)"""
    return np.ascontiguousarray(np.transpose(s, (0, 2, 1, 3)))


def to_oracle(g):
    return np.ascontiguousarray(np.transpose(g, (0, 2, 1, 3)))


def rand_fields(o, seed, amp=1.0, project=True):
    s = synthetic.random_coeffs((3, o.Kx, o.Ny, o.N), seed=seed, scale=amp)
    if project:
        s = o.state(o.project(o.pencils(s)))
    return s


def F_T(o, Fe):
    N = o.N
    return np.stack([np.linalg.solve(o.SS, np.moveaxis(Fe[..., f * N:(f + 1) * N], -1, 0).reshape(N, -1))
                     .reshape((N, o.Kx, o.Ny)).transpose(1, 2, 0) for f in range(3)])


def vjp_T(o, X, fbar):
    """(dF_T/dX)^dagger fbar = F_vjp(X, Y) with the C^(2) rows of Y = S1S0^-T fbar."""
    N = o.N
    Y = np.zeros((o.Kx, o.Ny, o.nvar), complex)
    for f in range(3):
        Y[..., f * N:(f + 1) * N] = np.linalg.solve(o.SS.T, fbar[f].reshape(-1, N).T).T.reshape(o.Kx, o.Ny, N)
    return o.state(o.F_vjp(X, Y))


def step_solve(o, v, a0, transpose=False):
    """P (prognostic part of (a0 M + L)^-1 [S1S0 v; 0]) or its adjoint map."""
    N = o.N
    if not transpose:
        R = np.zeros((o.Kx, o.Ny, o.nvar), complex)
        for f in range(3):
            R[..., f * N:(f + 1) * N] = v[f] @ o.SS.T
        return o.state(o.project(o.solve(a0, 1.0, R)))
    Y = o.solve_t(a0, 1.0, o.project(o.pencils(v)))
    return np.stack([Y[..., f * N:(f + 1) * N] @ o.SS for f in range(3)])


def _zc(shape):
    return torch.zeros(shape, dtype=torch.complex128, device="cuda")


@pytest.mark.parametrize("Nx,Ny,Nz", SMALL)
def test_transforms(Nx, Ny, Nz):
    from paper_2506_14792_gb300 import spadj
    o = oco.Couette(Nx, Ny, Nz, RE, pencils=False)
    p = gpu_problem(Nx, Ny, Nz)
    c = synthetic.random_coeffs((o.Kx, o.Ny, o.N), seed=Nx + Ny)
    g = np.random.default_rng(Nz).standard_normal((o.Mx, o.My, o.Mz))
    cg = dev(np.ascontiguousarray(c.transpose(1, 0, 2)))
    gg = dev(np.ascontiguousarray(g.transpose(2, 1, 0)))
    og = torch.zeros((o.Mz, o.My, o.Mx), dtype=torch.float64, device="cuda")
    oc = _zc((o.Ny, o.Kx, o.N))
    p.transform(spadj.C2G, cg, og)
    assert rel_err(host(og).transpose(2, 1, 0), o.c2g(c)) < 1e-13
    p.transform(spadj.G2C_ADJ, cg, og)
    assert rel_err(host(og).transpose(2, 1, 0), o.g2c_adj(c)) < 1e-13
    p.transform(spadj.G2C, gg, oc)
    assert rel_err(host(oc).transpose(1, 0, 2), o.g2c(g)) < 1e-13
    p.transform(spadj.C2G_ADJ, gg, oc)
    assert rel_err(host(oc).transpose(1, 0, 2), o.c2g_adj(g)) < 1e-13


@pytest.mark.parametrize("Nx,Ny,Nz", SMALL)
def test_F_jvp_vjp(Nx, Ny, Nz):
    o = oco.Couette(Nx, Ny, Nz, RE, pencils=False)
    p = gpu_problem(Nx, Ny, Nz)
    s, d = rand_fields(o, 1), rand_fields(o, 2)
    X = o.pencils(s)
    out = _zc((3, o.Ny, o.Kx, o.N))
    p.eval_F(dev(to_gpu(s)), out)
    assert rel_err(to_oracle(host(out)), F_T(o, o.F(X))) < 1e-12
    p.eval_F_jvp(dev(to_gpu(s)), dev(to_gpu(d)), out)
    assert rel_err(to_oracle(host(out)), F_T(o, o.F_jvp(X, o.pencils(d)))) < 1e-12
    p.eval_F_vjp(dev(to_gpu(s)), dev(to_gpu(d)), out)
    assert rel_err(to_oracle(host(out)), vjp_T(o, X, d)) < 1e-12


@pytest.mark.parametrize("Nx,Ny,Nz", SMALL)
def test_pencil_solve_and_adjoint(Nx, Ny, Nz):
    o = oco.Couette(Nx, Ny, Nz, RE)
    p = gpu_problem(Nx, Ny, Nz)
    v = rand_fields(o, 3, project=False)
    out = _zc((3, o.Ny, o.Kx, o.N))
    p.solve(dev(to_gpu(v)), out)
    assert rel_err(to_oracle(host(out)), step_solve(o, v, 1.5 / DT)) < 1e-12
    p.solve(dev(to_gpu(v)), out, transpose=True)
    assert rel_err(to_oracle(host(out)), step_solve(o, v, 1.5 / DT, transpose=True)) < 1e-12


@pytest.mark.parametrize("Nx,Ny,Nz", [(16, 6, 12), (32, 8, 16)])
def test_x_rows_per_cta_bitwise(Nx, Ny, Nz):
    """F and its VJP agree bitwise for 1, 2 and 4 x-FFT rows per CTA."""
    o = oco.Couette(Nx, Ny, Nz, RE, pencils=False)
    s, d = rand_fields(o, 21), rand_fields(o, 22)
    outs = []
    for nb in (1, 2, 4):
        p = gpu_problem(Nx, Ny, Nz)
        p.set_option(8, nb)
        f = _zc((3, o.Ny, o.Kx, o.N))
        v = _zc((3, o.Ny, o.Kx, o.N))
        p.eval_F(dev(to_gpu(s)), f)
        p.eval_F_vjp(dev(to_gpu(s)), dev(to_gpu(d)), v)
        outs.append((f, v))
    for f, v in outs[1:]:
        assert torch.equal(f, outs[0][0]) and torch.equal(v, outs[0][1])


@pytest.fixture(scope="module")
def traj_case():
    Nx, Ny, Nz, n = 16, 6, 12, 12
    o = oco.Couette(Nx, Ny, Nz, RE)
    u0 = synthetic.couette_ic(Nx, Ny, Nz, seed=5, norm=0.05)
    X0 = o.pencils(u0)
    J, g, X = oco.gain_gradient(o, X0, n, DT)
    return o, u0, X0, J, g, X, n


def test_forward_tangent_adjoint(traj_case):
    o, u0, X0, J, g, X, n = traj_case
    p = gpu_problem(o.Nx, o.Ny, o.Nz)
    x0 = dev(to_gpu(u0))
    xN = _zc(x0.shape)
    traj = _zc((n + 1,) + tuple(x0.shape))
    p.forward(n, x0, xN, traj)
    assert rel_err(to_oracle(host(xN)), o.state(X[-1])) < TOL
    assert rel_err(to_oracle(host(traj[n // 2])), o.state(X[n // 2])) < TOL
    d = rand_fields(o, 11, amp=0.05)
    dxN = _zc(x0.shape)
    p.tangent(n, x0, dev(to_gpu(d)), dxN)
    dX = imex.multistep_tangent(o, X, o.pencils(d), DT)
    assert rel_err(to_oracle(host(dxN)), o.state(dX[-1])) < TOL
    ybar = rand_fields(o, 12, project=False)
    gr = _zc(x0.shape)
    p.adjoint(n, traj, dev(to_gpu(ybar)), gr)
    want = imex.multistep_adjoint(o, X, lambda k: o.pencils(ybar) if k == n else None, DT)
    assert rel_err(to_oracle(host(gr)), o.state(want)) < TOL


def test_gain_gradient_and_checkpointing(traj_case):
    from paper_2506_14792_gb300 import spadj
    o, u0, X0, J, g, X, n = traj_case
    p = gpu_problem(o.Nx, o.Ny, o.Nz)
    x0 = dev(to_gpu(u0))
    gr = _zc(x0.shape)
    Jg = p.gradient(x0, n, gr, objective=spadj.SPADJ_OBJ_GAIN, ckpt_slots=0)
    assert abs(Jg[0] - J) < TOL * abs(J)
    assert rel_err(to_oracle(host(gr)), o.state(g)) < TOL
    for slots in (2, 3, 5):
        gc = _zc(x0.shape)
        Jc = p.gradient(x0, n, gc, objective=spadj.SPADJ_OBJ_GAIN, ckpt_slots=slots)
        assert Jc[0] == Jg[0]
        assert torch.equal(gc, gr), slots
    # two-level schedule: segment starts in page-locked host memory, device slots inside segments
    for slots, hslots in ((2, 3), (1, 4), (3, 2)):
        p.set_option(9, hslots)
        gc = _zc(x0.shape)
        Jc = p.gradient(x0, n, gc, objective=spadj.SPADJ_OBJ_GAIN, ckpt_slots=slots)
        assert Jc[0] == Jg[0]
        assert torch.equal(gc, gr), (slots, hslots)
    p.set_option(9, 0)


def test_energy_objective_and_vjp(traj_case):
    from paper_2506_14792_gb300 import spadj
    o, u0, X0, J, g, X, n = traj_case
    p = gpu_problem(o.Nx, o.Ny, o.Nz)
    x0 = dev(to_gpu(u0))
    gr = _zc(x0.shape)
    Je = p.gradient(x0, n, gr, objective=spadj.SPADJ_OBJ_ENERGY, ckpt_slots=4)
    want = imex.multistep_adjoint(o, X, lambda k: o.energy_grad(X[k]) if k == n else None, DT)
    assert abs(Je[0] - o.energy(X[-1])) < TOL * o.energy(X[-1])
    assert rel_err(to_oracle(host(gr)), o.state(want)) < TOL
    # cotangents injected at steps 0, 4 and n
    steps = [0, 4, n]
    seeds = [rand_fields(o, 40 + i, project=False) for i in range(3)]
    sd = dev(np.stack([to_gpu(s) for s in seeds]))
    gv = _zc(x0.shape)
    p.vjp(x0, n, steps, sd, gv, ckpt_slots=3)
    src = {k: o.pencils(s) for k, s in zip(steps, seeds)}
    want = imex.multistep_adjoint(o, X, lambda k: src.get(k), DT)
    assert rel_err(to_oracle(host(gv)), o.state(want)) < TOL


def test_energy_integral_objective(traj_case):
    """J = I(T) with dI/dt = E(X) integrated by the same scheme (the auxiliary ODE of
    Supplementary A.4) against the oracle's augmented system; checkpointed == store-all."""
    from paper_2506_14792_gb300 import spadj
    o, u0, X0, J, g, X, n = traj_case
    Jo, go, _ = imex.integral_gradient(o, X0, n, DT, o.energy, o.energy_grad)
    p = gpu_problem(o.Nx, o.Ny, o.Nz)
    x0 = dev(to_gpu(u0))
    gr = _zc(x0.shape)
    Jg = p.gradient(x0, n, gr, objective=spadj.SPADJ_OBJ_ENERGY_INTEGRAL)
    assert abs(Jg[0] - Jo) < TOL * abs(Jo)
    assert rel_err(to_oracle(host(gr)), o.state(go)) < TOL
    gc = _zc(x0.shape)
    Jc = p.gradient(x0, n, gc, objective=spadj.SPADJ_OBJ_ENERGY_INTEGRAL, ckpt_slots=3)
    assert Jc[0] == Jg[0] and torch.equal(gc, gr)


def test_linear_and_sbdf1():
    from paper_2506_14792_gb300 import spadj
    Nx, Ny, Nz, n = 8, 4, 8, 7
    for nonlinear, scheme, order in [(False, spadj.SPADJ_SBDF2, 2), (True, spadj.SPADJ_SBDF1, 1)]:
        o = oco.Couette(Nx, Ny, Nz, 300.0, nonlinear=nonlinear)
        p = gpu_problem(Nx, Ny, Nz, Re=300.0, dt=1e-2, nonlinear=nonlinear, scheme=scheme)
        u0 = synthetic.couette_ic(Nx, Ny, Nz, seed=9, norm=0.2)
        X = imex.multistep_forward(o, o.pencils(u0), n, 1e-2, order=order)
        E0, EN = o.energy(X[0]), o.energy(X[-1])
        dJ = lambda k: (o.energy_grad(X[k]) / E0 if k == n else (-(EN / E0 ** 2) * o.energy_grad(X[0])
                                                                  if k == 0 else None))
        want = imex.multistep_adjoint(o, X, dJ, 1e-2, order=order)
        gr = _zc((3, Ny, Nx // 2, Nz))
        Jg = p.gradient(dev(to_gpu(u0)), n, gr, objective=spadj.SPADJ_OBJ_GAIN)
        assert abs(Jg[0] - EN / E0) < TOL * EN / E0
        assert rel_err(to_oracle(host(gr)), o.state(want)) < TOL


# ---- full configuration 128 x 64 x 64, Re = 1000, dt = 5e-3 --------------------------------

FULL = (128, 64, 64)


@pytest.fixture(scope="module")
def full_case():
    p = gpu_problem(*FULL)
    u0 = synthetic.couette_ic(*FULL, seed=5)
    return p, u0


def test_full_explicit_term(full_case):
    p, u0 = full_case
    o = oco.Couette(*FULL, RE, pencils=False)
    out = _zc(to_gpu(u0).shape)
    p.eval_F(dev(to_gpu(u0)), out)
    assert rel_err(to_oracle(host(out)), F_T(o, o.F(o.pencils(u0)))) < 1e-12


def test_full_sampled_pencil_solves(full_case):
    p, u0 = full_case
    o = oco.Couette(*FULL, RE, pencils=False)
    N = o.N
    v = rand_fields(o, 21, project=False)
    out = _zc(to_gpu(v).shape)
    p.solve(dev(to_gpu(v)), out)
    got = to_oracle(host(out))
    p.solve(dev(to_gpu(v)), out, transpose=True)
    got_t = to_oracle(host(out))
    a0 = 1.5 / DT
    for m, j in [(1, 1), (5, 3), (63, 31), (17, 40), (30, 63), (2, 0)]:
        Mm, Lm = o.pencil_matrices(o.alpha[m], o.beta[j])
        A = a0 * Mm + Lm
        R = np.zeros(o.nvar, complex)
        for f in range(3):
            R[f * N:(f + 1) * N] = o.SS @ v[f, m, j]
        x = np.linalg.solve(A, R)[:3 * N]
        assert rel_err(got[:, m, j].ravel(), x) < 1e-11, (m, j)
        y = np.linalg.solve(A.conj().T, np.concatenate([v[:, m, j].ravel(), np.zeros(N + 7)]))
        want_t = np.concatenate([o.SS.T @ y[f * N:(f + 1) * N] for f in range(3)])
        assert rel_err(got_t[:, m, j].ravel(), want_t) < 1e-11, (m, j)


def test_full_trajectory_dot_and_fd(full_case):
    from paper_2506_14792_gb300 import spadj
    p, u0 = full_case
    n = 6
    x0 = dev(to_gpu(u0))
    o = oco.Couette(*FULL, RE, pencils=False)
    dx = dev(to_gpu(rand_fields(o, 31, amp=1e-5)))
    ybar = dev(to_gpu(rand_fields(o, 32)))
    traj = _zc((n + 1,) + tuple(x0.shape))
    xN = _zc(x0.shape)
    p.forward(n, x0, xN, traj)
    dxN = _zc(x0.shape)
    p.tangent(n, x0, dx, dxN)
    gr = _zc(x0.shape)
    p.adjoint(n, traj, ybar, gr)
    lhs = float(torch.sum((torch.conj(ybar) * dxN).real))
    rhs = float(torch.sum((torch.conj(gr) * dx).real))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
    g = _zc(x0.shape)
    J = p.gradient(x0, n, g, objective=spadj.SPADJ_OBJ_GAIN, ckpt_slots=3)[0]
    d = dev(to_gpu(synthetic.couette_ic(*FULL, seed=77, norm=1e-4)))
    eps = 1e-4
    Jp = p.gradient(x0 + eps * d, n, _zc(x0.shape), objective=spadj.SPADJ_OBJ_GAIN)[0]
    Jm = p.gradient(x0 - eps * d, n, _zc(x0.shape), objective=spadj.SPADJ_OBJ_GAIN)[0]
    fd = (Jp - Jm) / (2 * eps)
    ad = float(torch.sum((torch.conj(g) * d).real))
    assert abs(fd - ad) <= 1e-6 * abs(fd), (fd, ad, J)



@pytest.mark.parametrize("base", ["couette", "poiseuille"])
def test_resolvent_gains_all_pencils(base):
    """Energy-norm resolvent gains of every (kx, ky) pencil from the batched power iteration
    (forward and transposed pencil solves) against the oracle's dense generalised eigenproblem.
    Where the power iteration has converged ((lambda_next / lambda_1)^n_iter < 1e-20 by the
    oracle's spectrum) the gain must agree to 1e-10; elsewhere (the mean pencil at omega != 0,
    whose two slowest Stokes modes nearly tie) it must be a lower bound within 1e-2, as a
    Rayleigh quotient is."""
    import scipy.linalg as sla
    Nx, Ny, Nz, Re, n_iter = 8, 4, 16, 300.0, 120
    o = oco.Couette(Nx, Ny, Nz, Re, pencils=False, base=base)
    G3 = sla.block_diag(o.G, o.G, o.G)
    p = gpu_problem(Nx, Ny, Nz, Re=Re, base=base)
    for om in (0.0, 0.3):
        f = dev(to_gpu(synthetic.random_coeffs((3, o.Kx, o.Ny, o.N), seed=61)))
        gains = torch.zeros((Ny, Nx // 2), dtype=torch.float64, device="cuda")
        p.resolvent(om, n_iter, f, gains)
        gh = host(gains)
        for j in range(Ny):
            for m in range(o.Kx):
                if j == Ny // 2:
                    assert gh[j, m] == 0.0  # the unstored ky Nyquist row
                    continue
                R = oco.resolvent_matrix(o, o.alpha[m], o.beta[j], om)
                ev = sla.eigh(R.conj().T @ G3 @ R, G3, eigvals_only=True)[::-1]
                want = float(np.sqrt(ev[0]))
                assert abs(want - oco.resolvent_gain(o, o.alpha[m], o.beta[j], om)) <= 1e-12 * want
                nxt = next((e for e in ev[1:] if e < ev[0] * (1 - 1e-9)), 0.0)
                if (nxt / ev[0]) ** n_iter < 1e-20:
                    assert abs(gh[j, m] - want) <= 1e-10 * want, (om, j, m, gh[j, m], want)
                else:
                    assert want * (1 - 1e-2) <= gh[j, m] <= want * (1 + 1e-12), (om, j, m, gh[j, m], want)


def test_hessian_vector_product(traj_case):
    """Tangent-over-adjoint Hessian-vector product of J = E(X_N) against the oracle's."""
    o, u0, X0, J, g, X, n = traj_case
    v = synthetic.couette_ic(o.Nx, o.Ny, o.Nz, seed=91, norm=0.05)
    dX = imex.multistep_tangent(o, X, o.pencils(v), DT)
    want = imex.multistep_hvp(o, X, dX, lambda k: o.energy_grad(X[k]) if k == n else None,
                              lambda k: o.energy_grad(dX[k]) if k == n else None, DT)
    p = gpu_problem(o.Nx, o.Ny, o.Nz)
    hv = _zc(to_gpu(u0).shape)
    p.hvp(dev(to_gpu(u0)), dev(to_gpu(v)), n, hv)
    assert rel_err(to_oracle(host(hv)), o.state(want)) < TOL


def test_channel_flow_gain_gradient():
    """Plane Poiseuille (channel) profile: the SBDF2 gain gradient through the GPU path, store-all
    and checkpointed, against the oracle's."""
    from paper_2506_14792_gb300 import spadj
    Nx, Ny, Nz, n = 16, 6, 12, 10
    o = oco.Couette(Nx, Ny, Nz, RE, base="poiseuille")
    u0 = synthetic.couette_ic(Nx, Ny, Nz, seed=7, norm=0.05)
    J, g, X = oco.gain_gradient(o, o.pencils(u0), n, DT)
    p = gpu_problem(Nx, Ny, Nz, base="poiseuille")
    x0 = dev(to_gpu(u0))
    gr = _zc(x0.shape)
    Jg = p.gradient(x0, n, gr, objective=spadj.SPADJ_OBJ_GAIN, ckpt_slots=0)
    assert abs(Jg[0] - J) < TOL * abs(J)
    assert rel_err(to_oracle(host(gr)), o.state(g)) < TOL
    gc = _zc(x0.shape)
    p.gradient(x0, n, gc, objective=spadj.SPADJ_OBJ_GAIN, ckpt_slots=3)
    assert torch.equal(gc, gr)


@pytest.mark.parametrize("Nx,Ny,Nz,base", [(16, 6, 12, "couette"), (32, 8, 16, "couette"), (16, 8, 16, "poiseuille")])
def test_banded_and_dense_step_solves(Nx, Ny, Nz, base):
    """The two forms of the step solve (option 12: banded factors of the recombined pencil
    matrix, or the dense Phi) agree to rounding in both directions, the banded adjoint is the
    adjoint of the banded forward (dot test in the real inner product of the stored
    coefficients; P is an orthogonal projection for it), and a gain gradient agrees across the
    forms."""
    from paper_2506_14792_gb300 import spadj
    o = oco.Couette(Nx, Ny, Nz, RE, pencils=False)
    v = rand_fields(o, 31, project=False)
    w = rand_fields(o, 32, project=False)
    u0 = synthetic.couette_ic(Nx, Ny, Nz, seed=5, norm=0.05)
    res = {}
    for form in (1, 0):
        p = gpu_problem(Nx, Ny, Nz, base=base)
        p.set_option(12, form)
        a, b = _zc((3, o.Ny, o.Kx, o.N)), _zc((3, o.Ny, o.Kx, o.N))
        p.solve(dev(to_gpu(v)), a)
        p.solve(dev(to_gpu(w)), b, transpose=True)
        g = _zc((3, o.Ny, o.Kx, o.N))
        J = p.gradient(dev(to_gpu(u0)), 8, g, objective=spadj.SPADJ_OBJ_GAIN)
        res[form] = (host(a), host(b), host(g), J[0])
    assert rel_err(res[1][0], res[0][0]) < 1e-12
    assert rel_err(res[1][1], res[0][1]) < 1e-12
    # P (kx = 0 plane Hermitian in ky) is real-linear, not complex-linear: the identity holds for
    # the real inner product Re <a, b>
    lhs = np.vdot(to_gpu(w), res[1][0]).real
    rhs = np.vdot(res[1][1], to_gpu(v)).real
    assert abs(lhs - rhs) < 1e-12 * np.linalg.norm(to_gpu(w)) * np.linalg.norm(res[1][0])
    assert abs(res[1][3] - res[0][3]) < 1e-12 * abs(res[0][3])
    assert rel_err(res[1][2], res[0][2]) < 1e-11
