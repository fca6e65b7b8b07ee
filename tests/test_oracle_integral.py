"""Pins for time-integrated objectives (Supplementary A.4: the ODE dI/dt = g(X) is added to the
equation set and integrated by the same IMEX scheme; J = I(T)).

* Quadrature accuracy: for linear Burgers modes the energy decays as exp(-2 nu k^2 t), so
  I(T) = sum_k E_k (1 - exp(-2 nu k^2 T)) / (2 nu k^2); the scheme's I_N converges to it at
  second order in dt (SBDF2).
* Duality: I_N = sum_n s_n g(X_n) with the weights s_n of the scalar adjoint recurrence of the
  I-equation (the form the GPU path uses).
* Gradient (plane Couette, nonlinear): dot test between the augmented tangent and adjoint,
  central FD to 1e-6, Taylor rate 2.
"""
import numpy as np

import synthetic
from oracle import burgers, imex
from oracle import couette as co
from oracle.imex import inner


def test_integral_quadrature_second_order():
    N, nu, T = 16, 0.3, 0.5
    p = burgers.Burgers(N, nu, nonlinear=False)
    X0 = synthetic.burgers_ic(N, seed=3)[0]
    k = np.arange(N // 2)
    w = np.where(k == 0, 1.0, 2.0)
    E0 = 0.5 * p.length * w * np.abs(X0) ** 2           # energy per mode
    lam = 2 * nu * k ** 2
    exact = float(np.sum(np.where(lam > 0, E0 * (1 - np.exp(-lam * T)) / np.where(lam > 0, lam, 1), E0 * T)))
    errs = []
    for n in (40, 80, 160):
        J, _, _ = imex.integral_gradient(p, X0, n, T / n, p.energy, p.energy_grad)
        errs.append(abs(J - exact))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.15), (errs, rates)


def _weights(n_steps, dt, order=2):
    """s_n = sum_i c_i^{n+i} Y_{n+i} with Y_m the scalar adjoint of the I-equation (M = 1, L = 0):
    a_0^m Y_m = [m == N] - sum_i a_i^{m+i} Y_{m+i}."""
    Y = np.zeros(n_steps + 2 + order)
    co_ = [None] + [imex.sbdf_coeffs(m, order, dt) for m in range(1, n_steps + 1)]
    for m in range(n_steps, 0, -1):
        a, b, c = co_[m]
        r = 1.0 if m == n_steps else 0.0
        for i in (1, 2):
            if m + i <= n_steps and i < len(co_[m + i][0]):
                r -= co_[m + i][0][i] * Y[m + i]
        Y[m] = r / a[0]
    s = np.zeros(n_steps)
    for n in range(n_steps):
        for i in (1, 2):
            if n + i <= n_steps and i < len(co_[n + i][2]):
                s[n] += co_[n + i][2][i] * Y[n + i]
    return s


def test_integral_duality_weights():
    p = co.Couette(8, 6, 10, 300.0)
    X0 = p.pencils(synthetic.couette_ic(8, 6, 10, seed=5, norm=0.3))
    n, dt = 17, 2e-2
    J, _, V = imex.integral_gradient(p, X0, n, dt, p.energy, p.energy_grad)
    s = _weights(n, dt)
    assert abs(J - sum(s[k] * p.energy(V[k].X) for k in range(n))) < 1e-14 * abs(J)


def test_integral_gradient_dot_fd_taylor():
    p = co.Couette(8, 6, 10, 300.0)
    X0 = p.pencils(synthetic.couette_ic(8, 6, 10, seed=5, norm=0.3))
    n, dt = 20, 2e-2
    J, g, V = imex.integral_gradient(p, X0, n, dt, p.energy, p.energy_grad)
    aug = imex.IntegralObjective(p, p.energy, p.energy_grad)
    rng = np.random.default_rng(4)
    d = p.project(rng.standard_normal(X0.shape) + 1j * rng.standard_normal(X0.shape))
    dV = imex.multistep_tangent(aug, V, imex.Aug(d, 0.0), dt)
    assert abs(dV[-1].I.real - inner(g, d)) <= 1e-12 * abs(inner(g, d))
    Jf = lambda x: imex.integral_gradient(p, x, n, dt, p.energy, p.energy_grad)[0]
    for s in range(4):
        dd = p.pencils(synthetic.couette_ic(8, 6, 10, seed=200 + s, norm=1.0))
        eps = 1e-5 * np.linalg.norm(X0) / np.linalg.norm(dd)
        fd = (Jf(X0 + eps * dd) - Jf(X0 - eps * dd)) / (2 * eps)
        assert abs(fd - inner(g, dd)) <= 1e-6 * abs(fd)
    dd = p.pencils(synthetic.couette_ic(8, 6, 10, seed=300, norm=1.0)) * 0.3 * np.linalg.norm(X0)
    rem = [abs(Jf(X0 + e * dd) - J - e * inner(g, dd)) for e in (0.2, 0.1, 0.05, 0.025)]
    rates = np.log2(np.array(rem[:-1]) / np.array(rem[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.1), rates
