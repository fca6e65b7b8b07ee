"""GPU tests of the one-step C-ABI entry points (spadj_step_forward, spadj_step_tangent,
spadj_step_adjoint): chained one step at a time they reproduce the library's own sweeps bit for
bit (the same kernels on the same data) and the FP64 oracle to the parity bar.

The adjoint chain is the same for every scheme: y = NULL; for n = N..0: y = step_adjoint(n, X_n,
y, dJ/dX_n); dJ/dX_0 = the first state block of y (eq. IMEX_adjoint for the multistep schemes,
the RK adjoint for the Runge-Kutta schemes, Supplementary A.4)."""
import numpy as np
import pytest

import synthetic
from oracle import burgers as obur
from oracle import couette as oco
from oracle import imex
from oracle import rayleigh_benard as orb
from tests.gpu_util import TOL, dev, host, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _zeros(n):
    return torch.zeros(n, dtype=torch.float64, device="cuda")


def _flat(t):
    return (torch.view_as_real(t) if t.is_complex() else t).reshape(-1)


def _chain(p, x0, n_steps, dx0=None):
    """Forward (and tangent) chains of restart states; returns the list of X_n and, with dx0,
    the final tangent restart state."""
    ns, m = p.state_len(0), p.state_len(4)
    s = _zeros(m)
    s[:ns] = _flat(x0)
    ds = None
    if dx0 is not None:
        ds = _zeros(m)
        ds[:ns] = _flat(dx0)
    X = [s[:ns].clone()]
    for n in range(n_steps):
        if ds is not None:
            nd = _zeros(m)
            p.step_tangent(n, s, ds, nd)
            ds = nd
        nxt = _zeros(m)
        p.step_forward(n, s, nxt)
        s = nxt
        X.append(s[:ns].clone())
    return X, ds


def _adjoint_chain(p, X, seed_N, srcs=None):
    ns, m = p.state_len(0), p.state_len(5)
    y = None
    for n in range(len(X) - 1, -1, -1):
        src = seed_N if n == len(X) - 1 else (srcs.get(n) if srcs else None)
        out = _zeros(m)
        p.step_adjoint(n, X[n], y, out, src=src)
        y = out
    return y[:ns]


def _check_problem(p, x0, dx0, n_steps, slots, tangent_bitwise=True):
    """Step chains vs the sweeps of the same problem, bitwise.  (The Rayleigh-Benard tangent sweep
    recomputes its primal stages with the unfused column kernels, whose fold sums in another order
    than the fused forward step: there the step tangent agrees with it to rounding.)"""
    ns = p.state_len(0)
    X, ds = _chain(p, x0, n_steps, dx0)
    xN = _zeros(ns)
    p.forward(n_steps, x0.reshape(-1), xN)
    assert torch.equal(X[-1], xN)
    dxN = _zeros(ns)
    p.tangent(n_steps, x0.reshape(-1), dx0.reshape(-1), dxN)
    if tangent_bitwise:
        assert torch.equal(ds[:ns], dxN)
    else:
        assert rel_err(host(ds[:ns]), host(dxN)) < 1e-12
    Jd = _zeros(p.desc.batch)
    seed = _zeros(ns)
    p.objective(X[-1], Jd, seed)
    g_step = _adjoint_chain(p, X, seed)
    g = _zeros(ns)
    J = p.gradient(x0.reshape(-1), n_steps, g, ckpt_slots=slots)
    assert np.array_equal(J, host(Jd))
    assert torch.equal(g_step, g)
    return X, host(g_step)


def test_rb_steps_equal_sweeps_and_oracle():
    from tests.rb_util import gpu_problem
    Nx, Nz, dt, n = 16, 12, 1e-2, 10
    o = orb.RayleighBenard(Nx, Nz, 1e6)
    s0 = synthetic.rb_ic(Nx, Nz, seed=2, amp=0.3)
    d0 = synthetic.rb_ic(Nx, Nz, seed=5, amp=0.3)
    p = gpu_problem(Nx, Nz, dt=dt)
    assert p.state_len(4) == p.state_len(5) == p.state_len(0)
    X, g = _check_problem(p, dev(s0), dev(d0), n, slots=3, tangent_bitwise=False)
    Jo, go, Xo, _ = orb.gradient(o, o.pencils(s0), n, dt)
    assert rel_err(host(X[-1]).view(np.complex128).reshape(3, Nx // 2, Nz), o.state(Xo[-1])) < TOL
    assert rel_err(g.view(np.complex128).reshape(3, Nx // 2, Nz), o.state(go)) < TOL


def test_rb_steps_full_size_rk443_and_schedule():
    """256 x 64: RK222 with a step-size schedule (each step its own operators) and ARS(4,4,3)."""
    from paper_2506_14792_gb300 import spadj
    from tests.rb_util import gpu_problem
    Nx, Nz, n = 256, 64, 6
    s0 = dev(synthetic.rb_ic(Nx, Nz, seed=2, amp=1e-3))
    d0 = dev(synthetic.rb_ic(Nx, Nz, seed=7, amp=1.0))
    p = gpu_problem(Nx, Nz, dt=1e-3)
    p.set_dt_schedule([1e-3, 5e-4, 1e-3, 5e-4, 1e-3, 5e-4])
    _check_problem(p, s0, d0, n, slots=3, tangent_bitwise=False)
    q = gpu_problem(Nx, Nz, dt=1e-3, scheme=spadj.SPADJ_RK443)
    _check_problem(q, s0, d0, n, slots=2)


def test_couette_steps_equal_sweeps_and_oracle():
    from paper_2506_14792_gb300 import spadj
    Nx, Ny, Nz, dt, n = 8, 4, 8, 5e-3, 6
    o = oco.Couette(Nx, Ny, Nz, 1000.0)
    u0 = synthetic.couette_ic(Nx, Ny, Nz, seed=5, norm=0.05)
    du = synthetic.couette_ic(Nx, Ny, Nz, seed=6, norm=0.05)
    to_gpu = lambda s: np.ascontiguousarray(np.transpose(s, (0, 2, 1, 3)))
    p = spadj.Problem(spadj.SPADJ_COUETTE3D, spadj.SPADJ_SBDF2, [Nx, Ny, Nz], [4 * np.pi, 2 * np.pi], [1000.0], dt)
    ns = p.state_len(0)
    assert p.state_len(4) == 3 * ns and p.state_len(5) == 2 * ns
    X, g = _check_problem(p, dev(to_gpu(u0)), dev(to_gpu(du)), n, slots=3)
    # energy objective vs the oracle's multistep adjoint
    Xo = imex.multistep_forward(o, o.pencils(u0), n, dt)
    go = imex.multistep_adjoint(o, Xo, lambda k: o.energy_grad(Xo[k]) if k == n else None, dt)
    to_or = lambda a: np.transpose(a.view(np.complex128).reshape(3, Ny, Nx // 2, Nz), (0, 2, 1, 3))
    assert rel_err(to_or(host(X[-1])), o.state(Xo[-1])) < TOL
    assert rel_err(to_or(g), o.state(go)) < TOL
    # the gain objective: its explicit X_0 term enters the chain as the source at n = 0
    Jg, gg, _ = oco.gain_gradient(o, o.pencils(u0), n, dt)
    E0, EN = o.energy(o.pencils(u0)), o.energy(Xo[-1])
    Jd, e0, seedN, seed0 = _zeros(1), _zeros(1), _zeros(ns), _zeros(ns)
    p.objective(X[-1], Jd, seedN)
    p.objective(X[0], e0, seed0)
    src = {0: seed0 * (-EN / E0 ** 2)}
    gs = _adjoint_chain(p, X, seedN / E0, src)
    assert rel_err(to_or(host(gs)), o.state(gg)) < TOL


@pytest.mark.parametrize("scheme,n", [(2, 40), (5, 30)])
def test_burgers_steps_equal_sweeps_and_oracle(scheme, n):
    from paper_2506_14792_gb300 import spadj
    N, B, dt = 64, 3, 1e-3
    order = {2: 2, 5: 4}[scheme]
    p = spadj.Problem(spadj.SPADJ_BURGERS1D, scheme, [N], [2 * np.pi], [0.01], dt, batch=B)
    ns = p.state_len(0)
    assert p.state_len(4) == (2 * order - 1) * ns and p.state_len(5) == order * ns
    X0 = synthetic.burgers_ic(N, batch=B, seed=1)
    dX0 = synthetic.burgers_ic(N, batch=B, seed=4)
    X, g = _check_problem(p, dev(X0), dev(dX0), n, slots=4)
    o = obur.Burgers(N, 0.01)
    gview = g.view(np.complex128).reshape(B, N // 2)
    for b in range(B):
        Jo, go, _ = obur.gradient(o, X0[b], n, dt, order=order)
        assert rel_err(gview[b], go) < TOL


def test_burgers_checkpointed_gradient_equals_store_all():
    """Binomial schedule over device slots holding full restart states (X_n, X_{n-1}, F(X_{n-1})),
    and the two-level schedule with host slots: bitwise equal to the store-all sweep."""
    from paper_2506_14792_gb300 import spadj
    N, B, dt, n = 256, 7, 1e-3, 120
    X0 = dev(synthetic.burgers_ic(N, batch=B, seed=1))
    for scheme in (spadj.SPADJ_SBDF2, spadj.SPADJ_SBDF3):
        p = spadj.Problem(spadj.SPADJ_BURGERS1D, scheme, [N], [2 * np.pi], [0.01], dt, batch=B)
        ref = _zeros(p.state_len(0))
        J = p.gradient(X0, n, ref, ckpt_slots=0)
        for slots, hs in ((2, 0), (5, 0), (16, 0), (3, 4), (1, 6)):
            p.set_option(9, hs)
            g = _zeros(p.state_len(0))
            Jc = p.gradient(X0, n, g, ckpt_slots=slots)
            assert np.array_equal(Jc, J)
            assert torch.equal(g, ref), (scheme, slots, hs)
        p.set_option(9, 0)
        # injected cotangents (spadj_vjp) at several steps
        seeds = dev(synthetic.random_coeffs((3, B, N // 2), seed=3))
        ga, gb = _zeros(p.state_len(0)), _zeros(p.state_len(0))
        p.vjp(X0, n, [n, 40, 7], seeds, ga, ckpt_slots=0)
        p.vjp(X0, n, [n, 40, 7], seeds, gb, ckpt_slots=4)
        assert torch.equal(ga, gb)


def test_step_argument_errors():
    from paper_2506_14792_gb300 import spadj
    from tests.rb_util import gpu_problem
    p = gpu_problem(16, 12)
    a, b = _zeros(p.state_len(4)), _zeros(p.state_len(4))
    with pytest.raises(spadj.SpadjError) as e:
        p.step_forward(-1, a, b)
    assert e.value.status == spadj.SPADJ_ERR_INVALID
    L = spadj.lib()
    import ctypes
    st = L.spadj_step_forward(p.h, 0, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()))
    assert st == spadj.SPADJ_ERR_INVALID
    st = L.spadj_step_adjoint(p.h, 0, ctypes.c_void_p(a.data_ptr()), None, None, ctypes.c_void_p(b.data_ptr()),
                              ctypes.c_void_p(b.data_ptr()))
    assert st == spadj.SPADJ_ERR_INVALID  # gp_accum on a problem without parameters
    k = spadj.Problem(spadj.SPADJ_KOLMOGOROV2D, spadj.SPADJ_SBDF2, [16], [2 * np.pi], [100.0], 1e-3)
    assert k.state_len(4) == 3 * k.state_len(0) and k.state_len(5) == 2 * k.state_len(0)
    ka, kb = _zeros(k.state_len(4)), _zeros(k.state_len(4))
    st = L.spadj_step_tangent(k.h, 0, ctypes.c_void_p(ka.data_ptr()), ctypes.c_void_p(ka.data_ptr()),
                              ctypes.c_void_p(kb.data_ptr()))
    assert st == spadj.SPADJ_ERR_UNSUPPORTED  # the Kolmogorov batch has no tangent sweep
    e = spadj.Problem(spadj.SPADJ_SHEAR_EVP, 0, [0, 0, 16], [0.0], [1.0], 0.0, batch=2)
    assert e.state_len(4) == 0
    st = L.spadj_step_forward(e.h, 0, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()))
    assert st == spadj.SPADJ_ERR_UNSUPPORTED
