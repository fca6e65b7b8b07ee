"""GPU closure (BF16-operand / FP32-accumulate CNN inside the Kolmogorov F) against the FP64
oracle.  Stated tolerances: the closure correction and the gradients carry the BF16 operand
rounding of four stacked layers (about 2^-8 per operand), so they are compared at the
percent level, while the FP64 parts stay exact:
  * correction C(w; p) on the grid: max-norm relative error <= 3e-2
  * trajectory gradients w.r.t. the initial state and the 19105 parameters: <= 5e-2
  * zero parameters: the closure problem reproduces the plain solver bitwise."""
import numpy as np
import pytest

import synthetic
from oracle import cnn, imex
from oracle import kolmogorov as okol
from tests.gpu_util import dev, host, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, RE, DT = 64, 1000.0, 4e-3


def gpu_problem(batch, closure=True, dt=DT):
    from paper_2506_14792_gb300 import spadj
    return spadj.Problem(spadj.SPADJ_KOLMOGOROV2D, spadj.SPADJ_SBDF2, [N], [2 * np.pi], [RE, 0.0], dt, batch=batch,
                         closure=closure)


def test_param_count():
    p = gpu_problem(1)
    assert p.state_len(2) == cnn.n_params() == 19105


def test_closure_correction_matches_fp64():
    B = 3
    X = [okol.Kolmogorov(N, RE).project(synthetic.kolmogorov_ic(N, 300 + i)) for i in range(B)]
    params = synthetic.cnn_params(5, scale_out=1.0)
    p = gpu_problem(B)
    x = dev(np.concatenate([a.ravel() for a in X]))
    f0 = torch.zeros_like(x)
    f1 = torch.zeros_like(x)
    p.eval_F(x, f0)                       # zero parameters: plain F
    p.set_params(dev(params))
    p.eval_F(x, f1)
    C = host(f1 - f0).reshape(B, N // 2, N)
    o = okol.Kolmogorov(N, RE)
    net = cnn.CNN(params)
    for b in range(B):
        want = o.g2c(net.forward(o.c2g(X[b])))
        assert rel_err(C[b], want) < 3e-2


def test_zero_params_bitwise_plain():
    B, n = 2, 12
    X = dev(np.concatenate([okol.Kolmogorov(N, RE).project(synthetic.kolmogorov_ic(N, 400 + i)).ravel() for i in range(B)]))
    a = gpu_problem(B, closure=True)
    b = gpu_problem(B, closure=False)
    b.set_option(0, 0)
    oa, ob = torch.zeros_like(X), torch.zeros_like(X)
    a.forward(n, X, oa)
    b.forward(n, X, ob)
    assert torch.equal(oa, ob)


def test_closure_gradients_vs_fp64_oracle():
    from paper_2506_14792_gb300 import spadj
    B, nsteps, obs_steps = 2, 8, [4, 8]
    params = synthetic.cnn_params(6, scale_out=1.0)
    X0 = [okol.Kolmogorov(N, RE).project(synthetic.kolmogorov_ic(N, 500 + i)) for i in range(B)]
    tgt = [okol.Kolmogorov(N, RE).project(synthetic.kolmogorov_ic(N, 600 + i)) for i in range(B)]
    kmax = N // 2 - 1
    gx_ref, gp_ref, J_ref = [], 0, []
    for b in range(B):
        o = okol.Kolmogorov(N, RE, closure=cnn.CNN(params))
        X = imex.multistep_forward(o, X0[b], nsteps, DT)
        mask = o.lowpass_mask(kmax)
        ob = {n: mask * tgt[b] for n in obs_steps}
        J_ref.append(sum(o.misfit(X[n], ob[n], mask) for n in obs_steps))
        gx, gp = imex.multistep_adjoint_params(o, X, lambda n: o.misfit_grad(X[n], ob[n], mask) if n in ob else None, DT)
        gx_ref.append(gx)
        gp_ref = gp_ref + gp
    p = gpu_problem(B)
    p.set_params(dev(params))
    obs = np.stack([np.concatenate([(okol.Kolmogorov(N, RE).lowpass_mask(kmax) * tgt[b]).ravel() for b in range(B)])
                    for _ in obs_steps])
    p.set_observations(obs_steps, dev(obs), kmax)
    g = torch.zeros(B * (N // 2) * N, dtype=torch.complex128, device="cuda")
    gp = torch.zeros(cnn.n_params(), dtype=torch.float64, device="cuda")
    J = p.gradient(dev(np.concatenate([a.ravel() for a in X0])), nsteps, g, objective=spadj.SPADJ_OBJ_FOURDVAR, grad_p=gp)
    gh = host(g).reshape(B, N // 2, N)
    for b in range(B):
        assert abs(J[b] - J_ref[b]) <= 1e-2 * abs(J_ref[b])
        assert rel_err(gh[b], gx_ref[b]) < 5e-2
    assert rel_err(host(gp), gp_ref) < 5e-2
