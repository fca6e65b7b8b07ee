"""GPU closure (BF16-operand / FP32-accumulate CNN inside the Kolmogorov F) against the FP64
oracle.  The closure correction and the gradients carry the BF16 operand rounding of four stacked
layers (2^-9 relative per operand); measured on the GB300: correction 1.4-1.9e-3, J 1e-5,
dJ/dX_0 1e-5, dJ/dp 3.7e-3 (max-norm relative).  Bars (about 2.5-10x the measured errors, so a
dropped tap, channel block or reduction chunk, an error of several percent, fails):
  * correction C(w; p) on the grid: <= 5e-3
  * J and dJ/dX_0 of a trajectory objective: <= 1e-4; dJ/dp (19105 parameters): <= 1e-2
  * zero parameters: the closure problem reproduces the plain solver bitwise
  * each 32 -> 32 tensor-core convolution alone against the oracle's convolution of the same BF16
    operands (exact products and sums): <= 1e-5 (FP32 accumulation only)."""
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
    errs = []
    for b in range(B):
        want = o.g2c(net.forward(o.c2g(X[b])))
        errs.append(rel_err(C[b], want))
        assert errs[-1] < 5e-3
    print("closure correction vs FP64 oracle, max-norm relative error per member:", errs)


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
        assert abs(J[b] - J_ref[b]) <= 1e-4 * abs(J_ref[b])
        assert rel_err(gh[b], gx_ref[b]) < 1e-4
    assert rel_err(host(gp), gp_ref) < 1e-2
    print("closure gradients vs FP64 oracle: J", [abs(J[b] - J_ref[b]) / abs(J_ref[b]) for b in range(B)],
          "dJ/dX0", [rel_err(gh[b], gx_ref[b]) for b in range(B)], "dJ/dp", rel_err(host(gp), gp_ref))


def test_persistent_step_launches_equal_per_phase_launches():
    """The solver phases of a closure step as one persistent launch per step (option 0 = 1, the
    default: a member's B tiles start as soon as its own CA tiles are done) and as one launch per
    phase (option 0 = 0): the same arithmetic on every tile, so the forward states and the whole
    gradient (J, dJ/dX_0, dJ/dp) are bitwise equal."""
    from paper_2506_14792_gb300 import spadj
    B, nsteps, obs_steps = 3, 6, [3, 6]
    params = synthetic.cnn_params(7, scale_out=1.0)
    X0 = dev(np.concatenate([okol.Kolmogorov(N, RE).project(synthetic.kolmogorov_ic(N, 700 + i)).ravel()
                             for i in range(B)]))
    kmax = N // 2 - 1
    obs = np.stack([np.concatenate([(okol.Kolmogorov(N, RE).lowpass_mask(kmax) *
                                     okol.Kolmogorov(N, RE).project(synthetic.kolmogorov_ic(N, 800 + b + 10 * o))).ravel()
                                    for b in range(B)]) for o in range(len(obs_steps))])
    res = []
    for mode in (1, 0):
        p = gpu_problem(B)
        p.set_option(0, mode)
        p.set_params(dev(params))
        p.set_observations(obs_steps, dev(obs), kmax)
        xo = torch.zeros_like(X0)
        p.forward(nsteps, X0, xo)
        g = torch.zeros_like(X0)
        gp = torch.zeros(cnn.n_params(), dtype=torch.float64, device="cuda")
        J = p.gradient(X0, nsteps, g, objective=spadj.SPADJ_OBJ_FOURDVAR, grad_p=gp)
        res.append((xo, np.asarray(J), g, gp))
    (xa, Ja, ga, pa), (xb, Jb, gb, pb) = res
    assert torch.equal(xa, xb)
    assert np.array_equal(Ja, Jb)
    assert torch.equal(ga, gb)
    assert torch.equal(pa, pb)


def test_thin_weight_gradient_forms_agree():
    """The thin layers' weight and bias gradients (1 -> 32 and 32 -> 1) by the windowed kernel (all
    nine taps per CTA, the input window in registers; option 13 = 1, the default) and by one CTA
    per x offset (option 13 = 0): the same FP32 products summed in another order, so dJ/dp agrees to
    1e-5 (max-norm relative) and J and dJ/dX_0, which do not depend on them, are bitwise equal.  36
    modes on a 54 x 54 grid: row segments of 4 pixels with a ragged last lane of 2, bands of 13
    and 14 rows."""
    from paper_2506_14792_gb300 import spadj
    B, n, nsteps, obs_steps = 2, 36, 4, [2, 4]
    kmax = n // 2 - 1
    params = synthetic.cnn_params(9, scale_out=1.0)
    X0 = dev(np.concatenate([okol.Kolmogorov(n, RE).project(synthetic.kolmogorov_ic(n, 900 + i)).ravel()
                             for i in range(B)]))
    obs = np.stack([np.concatenate([(okol.Kolmogorov(n, RE).lowpass_mask(kmax) *
                                     okol.Kolmogorov(n, RE).project(synthetic.kolmogorov_ic(n, 950 + b + 10 * o))).ravel()
                                    for b in range(B)]) for o in range(len(obs_steps))])
    res = []
    for form in (1, 0):
        p = spadj.Problem(spadj.SPADJ_KOLMOGOROV2D, spadj.SPADJ_SBDF2, [n], [2 * np.pi], [RE, 0.0], DT, batch=B,
                          closure=True)
        p.set_option(13, form)
        p.set_params(dev(params))
        p.set_observations(obs_steps, dev(obs), kmax)
        g = torch.zeros_like(X0)
        gp = torch.zeros(cnn.n_params(), dtype=torch.float64, device="cuda")
        J = p.gradient(X0, nsteps, g, objective=spadj.SPADJ_OBJ_FOURDVAR, grad_p=gp)
        res.append((np.asarray(J), g, host(gp)))
    (Ja, ga, pa), (Jb, gb, pb) = res
    assert np.array_equal(Ja, Jb) and torch.equal(ga, gb)
    err = rel_err(pa, pb)
    print("thin weight-gradient forms: dJ/dp max-norm relative difference", err)
    assert err < 1e-5


def test_thin_output_forms_agree():
    """The thin layers' single-channel outputs (the 32 -> 1 forward into the closure term, the
    1 -> 32 input gradient into the grid cotangent) by the windowed kernel (a row segment per
    lane, the window of two channels per thread, the channel pairs added by a half-warp butterfly;
    option 14 = 1, the default) and by one thread per pixel with a 32-channel dot product per tap
    (option 14 = 0): the same FP32 products summed in another order, so the closure correction,
    J, dJ/dX_0 and dJ/dp agree to 1e-5 (max-norm relative).  36 modes on a 54 x 54 grid: row
    segments of 4 pixels with a ragged last lane of 2, bands of 6 and 7 rows."""
    from paper_2506_14792_gb300 import spadj
    B, n, nsteps, obs_steps = 2, 36, 4, [2, 4]
    kmax = n // 2 - 1
    params = synthetic.cnn_params(10, scale_out=1.0)
    X0 = dev(np.concatenate([okol.Kolmogorov(n, RE).project(synthetic.kolmogorov_ic(n, 960 + i)).ravel()
                             for i in range(B)]))
    obs = np.stack([np.concatenate([(okol.Kolmogorov(n, RE).lowpass_mask(kmax) *
                                     okol.Kolmogorov(n, RE).project(synthetic.kolmogorov_ic(n, 970 + b + 10 * o))).ravel()
                                    for b in range(B)]) for o in range(len(obs_steps))])
    res = []
    for form in (1, 0):
        p = spadj.Problem(spadj.SPADJ_KOLMOGOROV2D, spadj.SPADJ_SBDF2, [n], [2 * np.pi], [RE, 0.0], DT, batch=B,
                          closure=True)
        p.set_option(14, form)
        p.set_params(dev(params))
        f = torch.zeros_like(X0)
        p.eval_F(X0, f)
        p.set_observations(obs_steps, dev(obs), kmax)
        g = torch.zeros_like(X0)
        gp = torch.zeros(cnn.n_params(), dtype=torch.float64, device="cuda")
        J = p.gradient(X0, nsteps, g, objective=spadj.SPADJ_OBJ_FOURDVAR, grad_p=gp)
        res.append((host(f), np.asarray(J), host(g), host(gp)))
    (fa, Ja, ga, pa), (fb, Jb, gb, pb) = res
    errs = [rel_err(fa, fb), rel_err(Ja, Jb), rel_err(ga, gb), rel_err(pa, pb)]
    print("thin output forms: F, J, dJ/dX0, dJ/dp max-norm relative differences", errs)
    assert max(errs) < 1e-5


def _bf16(x):
    """float32 -> the nearest bfloat16 (round to nearest even), as float32 values and bit patterns."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = (((u >> 16) & 1) + 0x7FFF).astype(np.uint32)
    v = ((u + r) & np.uint32(0xFFFF0000)).view(np.float32)
    return v, (v.view(np.uint32) >> 16).astype(np.uint16)


@pytest.mark.parametrize("layer", [1, 2])
def test_tensor_core_convolution_vs_bf16_restated_oracle(layer):
    """The 32 -> 32 layers on the fifth-generation tensor cores (tcgen05.mma, FP32 accumulator in tensor
    memory), called alone through spadj_closure_conv in both operand-staging forms (halo tile with
    shifted descriptors, gather per tap): the pre-activation conv(x) + b and the input gradient
    conv^T(g) against the oracle's direct-sum convolution (oracle/cnn.py) applied to the same
    BF16-rounded operands with exact (FP64) products and sums: the only difference left is the FP32
    accumulation, so the bar is 1e-5 relative.  Three members of a 24 x 24 grid: 1728 pixels, 13.5
    tiles of 128 (a ragged last tile)."""
    from oracle import cnn as ocnn
    from paper_2506_14792_gb300 import spadj
    N, nb = 16, 3
    M = 3 * N // 2
    p = spadj.Problem(spadj.SPADJ_KOLMOGOROV2D, spadj.SPADJ_SBDF2, [N], [2 * np.pi], [RE, 0.0], 4e-3, batch=nb,
                      closure=True)
    prm = synthetic.cnn_params(11, scale_out=0.5)
    p.set_params(dev(prm))
    W, b = ocnn.unpack(prm)[layer]
    Wq = _bf16(W.astype(np.float32))[0].astype(np.float64)  # the library's FP64 -> FP32 -> BF16 rounding
    bq = b.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(layer)
    x = rng.uniform(-1.0, 1.0, (nb, 32, M, M)).astype(np.float32)  # oracle layout [member][c][x][y]
    xv, xbits = _bf16(x)
    inp = torch.from_numpy(np.ascontiguousarray(xbits.view(np.int16).transpose(0, 3, 2, 1))).cuda()  # [m][y][x][c]
    out = torch.zeros((nb, M, M, 32), dtype=torch.float32, device="cuda")
    res = {}
    for form in (2, 1):  # operand gathered per tap; operand staged once per tile (halo, the default)
        p.set_option(11, form)
        for mode in (0, 1):
            out.zero_()
            p.closure_conv(layer, mode, inp, out)
            res[(form, mode)] = host(out).copy()
            got = res[(form, mode)].transpose(0, 3, 2, 1)  # -> [m][o][x][y]
            for m in range(nb):
                xm = xv[m].astype(np.float64)
                ref = ocnn.conv(xm, Wq, bq) if mode == 0 else ocnn.conv_t(xm, Wq)
                err = np.max(np.abs(got[m] - ref)) / np.max(np.abs(ref))
                assert err < 1e-5, (layer, form, mode, m, err)
    for mode in (0, 1):  # the two staging forms issue the same MMAs in the same order
        assert np.max(np.abs(res[(1, mode)] - res[(2, mode)])) <= 1e-6 * np.max(np.abs(res[(2, mode)]))
    # the forward epilogue's activation (the exp-based tanh in FP32): 1 - tanh^2 of the kernel's own
    # FP32 pre-activations, against the FP64 tanh of the same values
    p.set_option(11, 1)
    out.zero_()
    p.closure_conv(layer, 2, inp, out)
    pre = res[(1, 0)].astype(np.float64)
    dact_err = np.max(np.abs(host(out) - (1.0 - np.tanh(pre) ** 2)))
    assert dact_err < 4e-6, dact_err
    # the warp-level mma.sync kernel computes the same input gradient
    p.set_option(11, 0)
    ref_tc = res[(1, 1)]
    out.zero_()
    p.closure_conv(layer, 1, inp, out)
    assert np.max(np.abs(host(out) - ref_tc)) <= 1e-5 * np.max(np.abs(ref_tc))
    p.set_option(11, 1)


def test_step_adjoint_accumulates_the_parameter_gradient():
    """With the learned closure, the chained spadj_step_adjoint calls add each step's parameter
    cotangent to gp_accum: the sum equals spadj_adjoint's grad_p over the stored trajectory (and the
    state gradient its grad_x0), bit for bit."""
    from paper_2506_14792_gb300 import spadj
    B, n = 2, 6
    p = gpu_problem(B)
    p.set_params(dev(synthetic.cnn_params(8, scale_out=1.0)))
    ns = p.state_len(0)
    X0 = dev(np.concatenate([okol.Kolmogorov(N, RE).project(synthetic.kolmogorov_ic(N, 700 + i)).ravel()
                             for i in range(B)]))
    traj = torch.zeros((n + 1, X0.numel()), dtype=torch.complex128, device="cuda")
    xN = torch.zeros_like(X0)
    p.forward(n, X0, xN, traj)
    yN = dev(np.concatenate([okol.Kolmogorov(N, RE).project(synthetic.kolmogorov_ic(N, 800 + i)).ravel()
                             for i in range(B)]))
    g_ref = torch.zeros_like(X0)
    gp_ref = torch.zeros(p.state_len(2), dtype=torch.float64, device="cuda")
    p.adjoint(n, traj, yN, g_ref, gp_ref)
    gp = torch.zeros_like(gp_ref)
    y = None
    for k in range(n, -1, -1):
        out = torch.zeros(p.state_len(5), dtype=torch.float64, device="cuda")
        p.step_adjoint(k, torch.view_as_real(traj[k]).reshape(-1).contiguous(), y, out,
                       src=torch.view_as_real(yN).reshape(-1) if k == n else None, gp_accum=gp)
        y = out
    assert torch.equal(y[:ns], torch.view_as_real(g_ref).reshape(-1))
    assert torch.equal(gp, gp_ref)


def test_weight_gradient_forms_agree():
    """The parameter gradient with the halo-staged ldmatrix weight gradient of the 32 -> 32 layers
    (default) equals the one with the per-tap mma.sync weight gradient (option 11 = 2, whose
    convolutions issue the same MMAs as the default ones) up to the FP32 summation order: 1e-5
    relative in max norm; the state gradient and J, which do not involve the weight gradient,
    agree to 1e-6 (the two convolution forms agree to that bar or better)."""
    from paper_2506_14792_gb300 import spadj
    B, n = 2, 4
    X0 = dev(np.concatenate([okol.Kolmogorov(N, RE).project(synthetic.kolmogorov_ic(N, 910 + i)).ravel()
                             for i in range(B)]))
    obs = torch.stack([X0 * (0.8 ** k) for k in range(1, n + 1)]).contiguous()
    out = {}
    for form in (1, 2):
        p = gpu_problem(B)
        p.set_option(11, form)
        p.set_params(dev(synthetic.cnn_params(9, scale_out=1.0)))
        p.set_observations(list(range(1, n + 1)), obs, N // 2 - 1)
        g = torch.zeros_like(X0)
        gp = torch.zeros(p.state_len(2), dtype=torch.float64, device="cuda")
        J = p.gradient(X0, n, g, objective=spadj.SPADJ_OBJ_FOURDVAR, grad_p=gp)
        out[form] = (J, host(g), host(gp))
    assert np.max(np.abs(out[1][0] - out[2][0]) / np.abs(out[2][0])) < 1e-6
    assert rel_err(out[1][1], out[2][1]) < 1e-6
    assert rel_err(out[1][2], out[2][2]) < 1e-5
    print("weight-gradient forms: dJ/dp relative difference", rel_err(out[1][2], out[2][2]))
