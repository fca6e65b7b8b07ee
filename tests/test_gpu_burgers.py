"""GPU parity for the Burgers path through the C-ABI against the FP64 oracle.

Sizes span several FFT passes (N = 16, 64, 256) and batches with a ragged tail;
the full configuration (N = 256, nu = 0.01, SBDF2, dt = 1e-3, 1000 steps, 16384
members) is checked on sampled members the oracle computes one by one.
"""
import numpy as np
import pytest

import synthetic
from oracle import burgers as obur
from oracle import fourier, imex
from tests.gpu_util import TOL, dev, host, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem(N, nu=0.01, dt=1e-3, batch=1, scheme=2, nonlinear=True):
    from paper_2506_14792_gb300 import spadj
    return spadj.Problem(spadj.SPADJ_BURGERS1D, scheme, [N], [2 * np.pi], [nu], dt, batch=batch, nonlinear=nonlinear)


def _adm(c):
    c = np.array(c, dtype=complex)
    c[..., 0] = c[..., 0].real
    return c


@pytest.mark.parametrize("N,B", [(16, 3), (64, 2), (256, 5)])
def test_transforms(N, B):
    from paper_2506_14792_gb300 import spadj
    p = _problem(N, batch=B)
    K, M = N // 2, 3 * N // 2
    c = _adm(synthetic.random_coeffs((B, K), seed=N))
    g = np.random.default_rng(N).standard_normal((B, M))
    out_g = torch.zeros((B, M), dtype=torch.float64, device="cuda")
    out_c = torch.zeros((B, K), dtype=torch.complex128, device="cuda")
    p.transform(spadj.C2G, dev(c), out_g)
    assert rel_err(host(out_g), fourier.c2g(c, M)) < 1e-13
    p.transform(spadj.G2C_ADJ, dev(c), out_g)
    assert rel_err(host(out_g), fourier.g2c_adj(c, M)) < 1e-13
    p.transform(spadj.G2C, dev(g), out_c)
    assert rel_err(host(out_c), fourier.g2c(g, K)) < 1e-13
    p.transform(spadj.C2G_ADJ, dev(g), out_c)
    assert rel_err(host(out_c), fourier.c2g_adj(g, K)) < 1e-13


@pytest.mark.parametrize("N,B", [(16, 2), (256, 3)])
def test_F_jvp_vjp(N, B):
    p = _problem(N, batch=B)
    o = obur.Burgers(N, 0.01)
    X = _adm(synthetic.random_coeffs((B, N // 2), seed=1))
    d = _adm(synthetic.random_coeffs((B, N // 2), seed=2))
    out = torch.zeros((B, N // 2), dtype=torch.complex128, device="cuda")
    p.eval_F(dev(X), out)
    assert rel_err(host(out), o.F(X)) < 1e-13
    p.eval_F_jvp(dev(X), dev(d), out)
    assert rel_err(host(out), o.F_jvp(X, d)) < 1e-13
    p.eval_F_vjp(dev(X), dev(d), out)
    assert rel_err(host(out), o.F_vjp(X, d)) < 1e-13


@pytest.mark.parametrize("N,B,nsteps", [(16, 1, 7), (64, 3, 50), (256, 2, 200)])
def test_forward_tangent_adjoint(N, B, nsteps):
    dt = 1e-3
    p = _problem(N, batch=B, dt=dt)
    o = obur.Burgers(N, 0.01)
    X0 = synthetic.burgers_ic(N, batch=B, seed=1)
    dX0 = _adm(synthetic.random_coeffs((B, N // 2), seed=9))
    traj = torch.zeros((nsteps + 1, B, N // 2), dtype=torch.complex128, device="cuda")
    xN = torch.zeros((B, N // 2), dtype=torch.complex128, device="cuda")
    p.forward(nsteps, dev(X0), xN, traj)
    Xo = imex.multistep_forward(o, X0, nsteps, dt)
    assert rel_err(host(xN), Xo[-1]) < TOL
    assert rel_err(host(traj), np.stack(Xo)) < TOL
    dxN = torch.zeros_like(xN)
    p.tangent(nsteps, dev(X0), dev(dX0), dxN)
    dXo = imex.multistep_tangent(o, Xo, dX0, dt)
    assert rel_err(host(dxN), dXo[-1]) < TOL
    yN = o.energy_grad(Xo[-1])
    g = torch.zeros_like(xN)
    p.adjoint(nsteps, traj, dev(yN), g)
    go = imex.multistep_adjoint(o, Xo, lambda n: yN if n == nsteps else None, dt)
    assert rel_err(host(g), go) < TOL


@pytest.mark.parametrize("order", [3, 4])
@pytest.mark.parametrize("N,B,nsteps", [(16, 2, 9), (256, 3, 120), (512, 2, 40)])
def test_higher_order_sbdf(order, N, B, nsteps):
    """SBDF3 / SBDF4 (lower-order first steps): forward, tangent, adjoint and the gradient of
    the energy against the oracle; the adjoint carries `order` pending cotangents."""
    from paper_2506_14792_gb300 import spadj
    dt = 1e-3
    scheme = {3: spadj.SPADJ_SBDF3, 4: spadj.SPADJ_SBDF4}[order]
    p = _problem(N, batch=B, dt=dt, scheme=scheme)
    o = obur.Burgers(N, 0.01)
    X0 = synthetic.burgers_ic(N, batch=B, seed=6)
    dX0 = _adm(synthetic.random_coeffs((B, N // 2), seed=16))
    traj = torch.zeros((nsteps + 1, B, N // 2), dtype=torch.complex128, device="cuda")
    xN = torch.zeros((B, N // 2), dtype=torch.complex128, device="cuda")
    p.forward(nsteps, dev(X0), xN, traj)
    Xo = imex.multistep_forward(o, X0, nsteps, dt, order)
    assert rel_err(host(traj), np.stack(Xo)) < TOL
    dxN = torch.zeros_like(xN)
    p.tangent(nsteps, dev(X0), dev(dX0), dxN)
    assert rel_err(host(dxN), imex.multistep_tangent(o, Xo, dX0, dt, order)[-1]) < TOL
    yN = _adm(synthetic.random_coeffs((B, N // 2), seed=17))
    g = torch.zeros_like(xN)
    p.adjoint(nsteps, traj, dev(yN), g)
    go = imex.multistep_adjoint(o, Xo, lambda n: yN if n == nsteps else None, dt, order)
    assert rel_err(host(g), go) < TOL
    gr = torch.zeros_like(xN)
    p.gradient(dev(X0), nsteps, gr)
    want = imex.multistep_adjoint(o, Xo, lambda n: o.energy_grad(Xo[-1]) if n == nsteps else None, dt, order)
    assert rel_err(host(gr), want) < TOL


def test_gpu_dot_test():
    N, B, nsteps, dt = 256, 4, 300, 1e-3
    p = _problem(N, batch=B, dt=dt)
    X0 = synthetic.burgers_ic(N, batch=B, seed=3)
    dX0 = _adm(synthetic.random_coeffs((B, N // 2), seed=4))
    yN = _adm(synthetic.random_coeffs((B, N // 2), seed=5))
    traj = torch.zeros((nsteps + 1, B, N // 2), dtype=torch.complex128, device="cuda")
    xN = torch.zeros((B, N // 2), dtype=torch.complex128, device="cuda")
    p.forward(nsteps, dev(X0), xN, traj)
    dxN = torch.zeros_like(xN)
    p.tangent(nsteps, dev(X0), dev(dX0), dxN)
    g = torch.zeros_like(xN)
    p.adjoint(nsteps, traj, dev(yN), g)
    for b in range(B):
        lhs = imex.inner(host(g)[b], dX0[b])
        rhs = imex.inner(yN[b], host(dxN)[b])
        assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_linear_diffusion_closed_form_gpu():
    N, nu, dt, nsteps = 32, 0.3, 1e-2, 60
    p = _problem(N, nu=nu, dt=dt, nonlinear=False)
    X0 = _adm(synthetic.random_coeffs((1, N // 2), seed=4))
    out = torch.zeros((1, N // 2), dtype=torch.complex128, device="cuda")
    p.forward(nsteps, dev(X0), out)
    k = np.arange(N // 2)
    z = nu * k ** 2 * dt
    x1 = X0[0] / (1 + z)
    disc = np.sqrt(4.0 - 2.0 * (1.5 + z) + 0j)
    r1, r2 = (2.0 + disc) / (2 * (1.5 + z)), (2.0 - disc) / (2 * (1.5 + z))
    Bc = (x1 - r1 * X0[0]) / (r2 - r1)
    want = (X0[0] - Bc) * r1 ** nsteps + Bc * r2 ** nsteps
    assert rel_err(host(out)[0], want) < 1e-13


def test_full_config_sampled_members():
    """N=256, nu=0.01, SBDF2 dt=1e-3, 1000 steps, 16384 members; gradient via spadj_gradient."""
    N, B, nsteps, dt = 256, 16384, 1000, 1e-3
    p = _problem(N, batch=B, dt=dt)
    X0 = synthetic.burgers_ic(N, batch=B, seed=1)
    g = torch.zeros((B, N // 2), dtype=torch.complex128, device="cuda")
    J = p.gradient(dev(X0), nsteps, g)
    gh = host(g)
    o = obur.Burgers(N, 0.01)
    for b in [0, 1, 8191, B - 1]:
        Jo, go, _ = obur.gradient(o, X0[b], nsteps, dt)
        assert abs(J[b] - Jo) <= TOL * abs(Jo)
        assert rel_err(gh[b], go) < TOL
    assert np.all(np.isfinite(J))


def test_invalid_arguments():
    from paper_2506_14792_gb300 import spadj
    with pytest.raises(spadj.SpadjError) as e:
        _problem(18)
    assert e.value.status == spadj.SPADJ_ERR_INVALID
    p = _problem(16)
    with pytest.raises(spadj.SpadjError):
        p.forward(-1, torch.zeros(8, dtype=torch.complex128, device="cuda"),
                  torch.zeros(8, dtype=torch.complex128, device="cuda"))


def test_variable_step_sbdf2_schedule():
    """Variable-step SBDF2 (spadj_set_dt_schedule): gradient against the oracle's SBDF weights built
    from the scheme's definition on the same nodes; a constant schedule reproduces the scalar-dt
    sweep bit for bit; checkpointed == store-all under the schedule; the step entry points follow the
    schedule."""
    from paper_2506_14792_gb300 import spadj
    N, B, n = 64, 3, 60
    sched = [2e-3 if (k // 9) % 2 == 0 else 7e-4 for k in range(n)]
    p = _problem(N, batch=B, dt=1e-3)
    X0 = synthetic.burgers_ic(N, batch=B, seed=1)
    g0 = torch.zeros((B, N // 2), dtype=torch.complex128, device="cuda")
    ref = torch.zeros_like(g0)
    J0 = p.gradient(dev(X0), n, ref)
    p.set_dt_schedule([1e-3] * n)
    J1 = p.gradient(dev(X0), n, g0)
    assert np.array_equal(J0, J1) and torch.equal(g0, ref)
    p.set_dt_schedule(sched)
    g = torch.zeros_like(g0)
    J = p.gradient(dev(X0), n, g)
    o = obur.Burgers(N, 0.01)
    for b in range(B):
        Jo, go, _ = obur.gradient(o, X0[b], n, sched)
        assert abs(J[b] - Jo) <= TOL * abs(Jo)
        assert rel_err(host(g)[b], go) < TOL
    gc = torch.zeros_like(g0)
    Jc = p.gradient(dev(X0), n, gc, ckpt_slots=5)
    assert np.array_equal(Jc, J) and torch.equal(gc, g)
    with pytest.raises(spadj.SpadjError):
        p.gradient(dev(X0), n + 1, gc)  # longer than the schedule
    q = _problem(N, batch=B, dt=1e-3, scheme=spadj.SPADJ_SBDF3)
    with pytest.raises(spadj.SpadjError) as e:
        q.set_dt_schedule(sched)
    assert e.value.status == spadj.SPADJ_ERR_UNSUPPORTED
