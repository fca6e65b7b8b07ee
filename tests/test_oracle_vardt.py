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
