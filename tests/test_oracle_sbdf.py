"""Pins for the higher-order multistep IMEX schemes SBDF3 and SBDF4 of the oracle.

* The weights built from the scheme's definition (backward differentiation for the implicit
  part, Lagrange extrapolation of F for the explicit part) reproduce the SBDF1 / SBDF2
  weights written out by hand.
* Local truncation error: one step from the exact history of y' = -(lam_I + lam_E) y, with
  lam_I implicit and F = -lam_E y explicit, errs by O(dt^(s+1)) for SBDF<s>; a wrong or
  dropped weight in either part lowers the order.
* The adjoint recurrence (eq. IMEX_adjoint) with s pending cotangents: dot test against the
  tangent and central finite differences on a nonlinear Burgers trajectory.
"""
import numpy as np
import pytest

import synthetic
from oracle import burgers, imex
from oracle.imex import inner


def test_definition_reproduces_sbdf1_and_sbdf2():
    for s in (1, 2):
        a, c = imex.sbdf_weights(s)
        a_h, _, c_h = imex.sbdf_coeffs(s, s, 1.0)
        assert [float(v) for v in a] == list(a_h) and [float(v) for v in c] == list(c_h)


@pytest.mark.parametrize("s", [1, 2, 3, 4])
def test_local_truncation_order(s):
    lam_i, lam_e = 1.3 + 0.7j, 0.4 - 0.9j
    y = lambda t: np.exp(-(lam_i + lam_e) * t)
    errs, dts = [], [0.08, 0.04, 0.02, 0.01]
    for dt in dts:
        a, b, c = imex.sbdf_coeffs(s, s, dt)
        t = s * dt
        rhs = sum(c[i] * (-lam_e * y(t - i * dt)) - a[i] * y(t - i * dt) for i in range(1, s + 1))
        yn = rhs / (a[0] + b[0] * lam_i)
        errs.append(abs(yn - y(t)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - (s + 1)) < 0.25), (s, errs, rates)


@pytest.mark.parametrize("order", [3, 4])
def test_adjoint_dot_test_and_fd(order):
    N, nu, dt, nsteps = 32, 0.02, 2e-3, 60
    prob = burgers.Burgers(N, nu)
    X0 = synthetic.burgers_ic(N, batch=1, seed=3)[0]
    J, g, X = burgers.gradient(prob, X0, nsteps, dt, order)
    for k in range(2):
        d = synthetic.random_coeffs(prob.K, seed=70 + k)
        d[0] = d[0].real
        dX = imex.multistep_tangent(prob, X, d, dt, order)
        assert abs(inner(g, d) - inner(prob.energy_grad(X[-1]), dX[-1])) <= 1e-12 * abs(inner(g, d))
        eps = 1e-5 * np.linalg.norm(X0) / np.linalg.norm(d)
        Jp = prob.energy(imex.multistep_forward(prob, X0 + eps * d, nsteps, dt, order)[-1])
        Jm = prob.energy(imex.multistep_forward(prob, X0 - eps * d, nsteps, dt, order)[-1])
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - inner(g, d)) <= 1e-6 * abs(fd)
