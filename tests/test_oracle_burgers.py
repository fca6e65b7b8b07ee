"""Pins for the Burgers oracle: multistep IMEX forward map, tangent and adjoint.

* F=0: every mode follows the exact discrete SBDF1->SBDF2 recurrence (closed form
  by the roots of the characteristic polynomial) and converges to exp(-nu k^2 t)
  at second order in dt (Supplementary A.4, eq. imex).
* Nonlinear forward: converges to the Cole-Hopf exact solution of viscous Burgers
  at second order in dt (fixes the sign and factor of -d/dx(u^2/2) and of nu).
* F_jvp equals the central difference of F exactly (F is quadratic); F_vjp is its
  transpose (brute-force Jacobian for a tiny size).
* Whole trajectory: dot test <dJ/dX_0, dX_0> = <dJ/dX_N, dX_N> between the adjoint
  (eq. IMEX_adjoint) and the tangent, central finite differences, Taylor remainder
  rate 2 (Supplementary C).
"""
import numpy as np
import pytest

import synthetic
from oracle import burgers, fourier, imex
from oracle.imex import inner


def _adm(c):
    c = np.array(c, dtype=complex)
    c[..., 0] = c[..., 0].real
    return c


def test_linear_diffusion_closed_form():
    N, nu, dt, nsteps = 32, 0.3, 1e-2, 60
    prob = burgers.Burgers(N, nu, nonlinear=False)
    X0 = _adm(synthetic.random_coeffs(N // 2, seed=4))
    X = imex.multistep_forward(prob, X0, nsteps, dt)
    z = nu * prob.k ** 2 * dt
    x1 = X0 / (1 + z)                                  # SBDF1 first step
    disc = np.sqrt(4.0 - 2.0 * (1.5 + z) + 0j)          # roots of (3/2+z) r^2 - 2 r + 1/2 = 0
    r1 = (2.0 + disc) / (2 * (1.5 + z))
    r2 = (2.0 - disc) / (2 * (1.5 + z))
    B = (x1 - r1 * X0) / (r2 - r1)
    A = X0 - B
    for n in [1, 2, 5, 30, nsteps]:
        want = A * r1 ** n + B * r2 ** n
        np.testing.assert_allclose(X[n], want, rtol=1e-13, atol=1e-15)


def test_linear_diffusion_second_order():
    N, nu, T = 16, 1.0, 0.5
    prob = burgers.Burgers(N, nu, nonlinear=False)
    X0 = np.zeros(N // 2, complex)
    X0[1] = 1.0
    errs = []
    for nsteps in [50, 100, 200]:
        X = imex.multistep_forward(prob, X0, nsteps, T / nsteps)
        errs.append(abs(X[-1][1] - np.exp(-nu * T)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.1), rates


def cole_hopf(x, t, nu, eps):
    e = eps * np.exp(-nu * t)
    return 2.0 * nu * e * np.sin(x) / (1.0 + e * np.cos(x))


def test_cole_hopf_exact_solution_and_order():
    N, nu, eps, T = 64, 0.1, 0.8, 0.4
    prob = burgers.Burgers(N, nu)
    xg = prob.grid_points()
    X0 = fourier.g2c(cole_hopf(xg, 0.0, nu, eps), prob.K)
    errs = []
    for nsteps in [40, 80, 160]:
        X = imex.multistep_forward(prob, X0, nsteps, T / nsteps)
        errs.append(np.max(np.abs(prob.to_grid(X[-1]) - cole_hopf(xg, T, nu, eps))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 1e-5
    assert np.all(np.abs(rates - 2.0) < 0.15), (errs, rates)


def test_F_bruteforce_and_jvp_vjp():
    N = 8
    prob = burgers.Burgers(N, 0.1)
    K, M = prob.K, prob.Mg
    X = _adm(synthetic.random_coeffs(K, seed=7))
    # brute force from explicit cos/sin matrices
    u = fourier.dense_c2g(K, M) @ fourier.to_real(X)
    what = fourier.from_real(fourier.dense_g2c(K, M) @ (0.5 * u * u))
    np.testing.assert_allclose(prob.F(X), -1j * prob.k * what, atol=1e-14)
    # JVP = exact central difference of a quadratic map
    for s in range(4):
        dX = _adm(synthetic.random_coeffs(K, seed=20 + s))
        h = 1e-3
        fd = (prob.F(X + h * dX) - prob.F(X - h * dX)) / (2 * h)
        np.testing.assert_allclose(prob.F_jvp(X, dX), fd, atol=1e-12)
    # VJP = transpose of the brute-force Jacobian
    Jm = np.zeros((2 * K, 2 * K))
    for i in range(2 * K):
        e = np.zeros(2 * K)
        e[i] = 1.0
        Jm[:, i] = fourier.to_real(prob.F_jvp(X, fourier.from_real(e)))
    for i in range(2 * K):
        e = np.zeros(2 * K)
        e[i] = 1.0
        np.testing.assert_allclose(fourier.to_real(prob.F_vjp(X, fourier.from_real(e))), Jm[i], atol=1e-13)


def test_energy_closed_form():
    prob = burgers.Burgers(16, 0.1)
    xg = prob.grid_points()
    X = fourier.g2c(np.cos(3 * xg), prob.K)
    assert abs(prob.energy(X) - np.pi / 2) < 1e-14
    X = fourier.g2c(2.0 + np.sin(xg), prob.K)
    assert abs(prob.energy(X) - 0.5 * (8 * np.pi + np.pi)) < 1e-13


@pytest.fixture(scope="module")
def traj():
    N, nu, dt, nsteps = 64, 0.01, 1e-3, 300
    prob = burgers.Burgers(N, nu)
    X0 = synthetic.burgers_ic(N, batch=1, seed=1)[0]
    J, g, X = burgers.gradient(prob, X0, nsteps, dt)
    return prob, X0, J, g, X, dt, nsteps


def test_dot_test_tangent_vs_adjoint(traj):
    prob, X0, J, g, X, dt, nsteps = traj
    for s in range(3):
        dX0 = _adm(synthetic.random_coeffs(prob.K, seed=100 + s))
        dX = imex.multistep_tangent(prob, X, dX0, dt)
        lhs = inner(g, dX0)
        rhs = inner(prob.energy_grad(X[-1]), dX[-1])
        assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_gradient_central_fd(traj):
    prob, X0, J, g, X, dt, nsteps = traj
    for s in range(8):
        d = _adm(synthetic.random_coeffs(prob.K, seed=200 + s))
        eps = 1e-5 * np.linalg.norm(X0) / np.linalg.norm(d)
        Jp = prob.energy(imex.multistep_forward(prob, X0 + eps * d, nsteps, dt)[-1])
        Jm = prob.energy(imex.multistep_forward(prob, X0 - eps * d, nsteps, dt)[-1])
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - inner(g, d)) <= 1e-6 * abs(fd)


def test_taylor_remainder_rate(traj):
    prob, X0, J, g, X, dt, nsteps = traj
    d = _adm(synthetic.random_coeffs(prob.K, seed=300))
    d *= 0.1 * np.linalg.norm(X0) / np.linalg.norm(d)
    eps = [1e-1, 5e-2, 2.5e-2, 1.25e-2]
    rem = []
    for e in eps:
        Je = prob.energy(imex.multistep_forward(prob, X0 + e * d, nsteps, dt)[-1])
        rem.append(abs(Je - J - e * inner(g, d)))
    rates = np.log2(np.array(rem[:-1]) / np.array(rem[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.05), rates


def test_imag_mean_mode_dead(traj):
    prob, X0, J, g, X, dt, nsteps = traj
    assert g[0].imag == 0.0
    X0b = X0.copy()
    X0b[0] += 0.3j
    Xb = imex.multistep_forward(prob, X0b, 5, dt)
    np.testing.assert_array_equal(Xb[-1], imex.multistep_forward(prob, X0, 5, dt)[-1])
