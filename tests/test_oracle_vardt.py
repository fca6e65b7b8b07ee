"""Pins for step-dependent timesteps in the oracle's Runge-Kutta IMEX forward, tangent and
adjoint (the stage operators are refactorised when the step size changes).

* A constant schedule reproduces the scalar-dt path exactly.
* Linear diffusion (F = 0) under a varying schedule: every mode is multiplied by the ARS(2,2,2)
  amplification factor of each step's own z_n = nu k^2 dt_n (closed form).
* Rayleigh-Benard gradient under a varying schedule: dot test against the tangent and central
  finite differences.
"""
import numpy as np

import synthetic
from oracle import burgers, imex
from oracle import rayleigh_benard as rb
from oracle.imex import inner

SCHEDULE = [1e-2, 1e-2, 4e-3, 4e-3, 4e-3, 7e-3, 1e-2, 2e-3]


def test_constant_schedule_equals_scalar_dt():
    p = rb.RayleighBenard(16, 12, 1e6)
    X0 = p.pencils(synthetic.rb_ic(16, 12, seed=2, amp=0.3))
    A, H = imex.rk222_tableaux()
    Xa, _ = imex.rk_forward(p, X0, 5, 5e-3, A, H)
    Xb, _ = imex.rk_forward(p, X0, 5, [5e-3] * 5, A, H)
    assert all(np.array_equal(a, b) for a, b in zip(Xa, Xb))


def test_linear_diffusion_closed_form_varying_steps():
    N, nu = 16, 0.3
    prob = burgers.Burgers(N, nu, nonlinear=False)
    X0 = synthetic.random_coeffs(N // 2, seed=8)
    X0[0] = X0[0].real
    A, H = imex.rk222_tableaux()
    X, _ = imex.rk_forward(prob, X0, len(SCHEDULE), SCHEDULE, A, H)
    g = imex.RK222_GAMMA
    want = X0.copy()
    for dt in SCHEDULE:
        z = nu * prob.k ** 2 * dt
        want = want * (1.0 - (1.0 - g) * z / (1.0 + g * z)) / (1.0 + g * z)
    np.testing.assert_allclose(X[-1], want, rtol=1e-13, atol=1e-16)


def test_rb_gradient_varying_steps():
    p = rb.RayleighBenard(16, 12, 1e6)
    X0 = p.pencils(synthetic.rb_ic(16, 12, seed=2, amp=0.3))
    n = len(SCHEDULE)
    for tab in (imex.rk222_tableaux(), imex.rk443_tableaux()):
        J, g, X, stages = rb.gradient(p, X0, n, SCHEDULE, tab)
        Jf = lambda X0_: p.kinetic_energy(imex.rk_forward(p, X0_, n, SCHEDULE, *tab)[0][-1])
        d = p.pencils(synthetic.rb_ic(16, 12, seed=61, amp=1.0))
        dX = imex.rk_tangent(p, stages, d, SCHEDULE, *tab)
        assert abs(inner(g, d) - inner(p.kinetic_energy_grad(X[-1]), dX[-1])) <= 1e-12 * abs(inner(g, d))
        eps = 1e-5 * np.linalg.norm(X0) / np.linalg.norm(d)
        fd = (Jf(X0 + eps * d) - Jf(X0 - eps * d)) / (2 * eps)
        assert abs(fd - inner(g, d)) <= 1e-6 * abs(fd)


# ---- variable-step SBDF2 (multistep schemes under a step-size schedule) -----------------------

def test_variable_sbdf2_weights_match_the_published_closed_form():
    """Weights built from the scheme's definition on the actual nodes equal the Wang-Ruuth closed
    form of variable-step SBDF2 (w = h_n / h_{n-1}): a0 = (1 + 2w)/((1 + w) h_n), a1 = -(1 + w)/h_n,
    a2 = w^2/((1 + w) h_n), c1 = 1 + w, c2 = -w."""
    for hn, hm in ((1e-2, 1e-2), (4e-3, 1e-2), (1e-2, 3e-3), (7e-3, 5e-3)):
        a, b, c = imex.sbdf_coeffs(2, 2, [hm, hn])
        w = hn / hm
        want_a = [(1 + 2 * w) / ((1 + w) * hn), -(1 + w) / hn, w * w / ((1 + w) * hn)]
        want_c = [0.0, 1 + w, -w]
        assert np.allclose(a, want_a, rtol=1e-14, atol=0)
        assert np.allclose(c, want_c, rtol=1e-14, atol=1e-15)
        assert list(b) == [1.0, 0.0, 0.0]
    a1, _, c1 = imex.sbdf_coeffs(1, 2, [4e-3])  # first step: backward/forward Euler of its own size
    assert np.allclose(a1, [1 / 4e-3, -1 / 4e-3], rtol=1e-15) and list(c1) == [0.0, 1.0]


def test_constant_schedule_sbdf2_equals_scalar_dt():
    prob = burgers.Burgers(32, 0.02)
    X0 = synthetic.burgers_ic(32, batch=1, seed=3)[0]
    Xa = imex.multistep_forward(prob, X0, 20, 2e-3)
    Xb = imex.multistep_forward(prob, X0, 20, [2e-3] * 20)
    assert max(np.max(np.abs(a - b)) for a, b in zip(Xa, Xb)) <= 1e-14 * np.max(np.abs(X0))


def test_variable_sbdf2_local_truncation_order():
    """One step from the exact history of y' = -(lam_I + lam_E) y on unequal steps (ratio 0.4):
    the error falls as h^3, as for a second-order method (a weight that ignored the ratio would
    lose an order)."""
    lam_i, lam_e = 1.3 + 0.7j, 0.4 - 0.9j
    y = lambda t: np.exp(-(lam_i + lam_e) * t)
    errs, hs = [], [0.08, 0.04, 0.02, 0.01]
    for h in hs:
        steps = [h, 0.4 * h]  # h_{n-1}, h_n
        a, b, c = imex.sbdf_coeffs(2, 2, steps)
        tn = sum(steps)
        ts = [tn, tn - steps[1], 0.0]
        rhs = sum(c[i] * (-lam_e * y(ts[i])) - a[i] * y(ts[i]) for i in (1, 2))
        errs.append(abs(rhs / (a[0] + b[0] * lam_i) - y(tn)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 3) < 0.25), (errs, rates)


def test_variable_sbdf2_burgers_adjoint_dot_test_and_fd():
    N, nu, nsteps = 32, 0.02, 40
    sched = [2e-3 if (n // 7) % 2 == 0 else 1e-3 for n in range(nsteps)]
    prob = burgers.Burgers(N, nu)
    X0 = synthetic.burgers_ic(N, batch=1, seed=3)[0]
    J, g, X = burgers.gradient(prob, X0, nsteps, sched)
    for k in range(2):
        d = synthetic.random_coeffs(prob.K, seed=80 + k)
        d[0] = d[0].real
        dX = imex.multistep_tangent(prob, X, d, sched)
        assert abs(inner(g, d) - inner(prob.energy_grad(X[-1]), dX[-1])) <= 1e-12 * abs(inner(g, d))
        eps = 1e-5 * np.linalg.norm(X0) / np.linalg.norm(d)
        Jp = prob.energy(imex.multistep_forward(prob, X0 + eps * d, nsteps, sched)[-1])
        Jm = prob.energy(imex.multistep_forward(prob, X0 - eps * d, nsteps, sched)[-1])
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - inner(g, d)) <= 1e-6 * abs(fd)
