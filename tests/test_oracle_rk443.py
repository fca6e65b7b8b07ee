"""Pins for the third-order Runge-Kutta IMEX scheme ARS(4,4,3) of the oracle.

* Both tableaux are consistent (row sums are the common stage times) and share them.
* Third order on the Cole-Hopf exact solution of viscous Burgers (explicit nonlinear term,
  implicit diffusion): a wrong entry in either tableau lowers the rate.
* The RK adjoint (Supplementary A.4) with four stages on a Rayleigh-Benard trajectory: dot
  test against the tangent and central finite differences of the kinetic energy.
"""
import numpy as np

import synthetic
from oracle import burgers, fourier, imex
from oracle import rayleigh_benard as rb
from oracle.imex import inner


def test_tableaux_consistent():
    A, H = imex.rk443_tableaux()
    np.testing.assert_allclose(A.sum(axis=1), H.sum(axis=1), rtol=0, atol=1e-15)
    np.testing.assert_allclose(A.sum(axis=1), [0.0, 0.5, 2.0 / 3.0, 0.5, 1.0], rtol=0, atol=1e-15)
    assert np.all(np.diag(H)[1:] == 0.5) and np.all(H[:, 0] == 0.0)
    assert np.all(np.triu(A) == 0.0) and np.all(np.triu(H, 1) == 0.0)


def test_third_order_cole_hopf():
    from tests.test_oracle_burgers import cole_hopf
    N, nu, eps, T = 64, 0.1, 0.8, 0.4
    prob = burgers.Burgers(N, nu)
    xg = prob.grid_points()
    X0 = fourier.g2c(cole_hopf(xg, 0.0, nu, eps), prob.K)
    A, H = imex.rk443_tableaux()
    errs = []
    for nsteps in [20, 40, 80, 160]:
        X, _ = imex.rk_forward(prob, X0, nsteps, T / nsteps, A, H)
        errs.append(np.max(np.abs(prob.to_grid(X[-1]) - cole_hopf(xg, T, nu, eps))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 3.0) < 0.15), (errs, rates)


def test_rb_adjoint_dot_test_and_fd():
    p = rb.RayleighBenard(16, 12, 1e6)
    X0 = p.pencils(synthetic.rb_ic(16, 12, seed=2, amp=0.3))
    dt, nsteps = 1e-2, 12
    tab = imex.rk443_tableaux()
    J, g, X, stages = rb.gradient(p, X0, nsteps, dt, tab)
    Jf = lambda X0_: p.kinetic_energy(imex.rk_forward(p, X0_, nsteps, dt, *tab)[0][-1])
    for s in range(2):
        d = p.pencils(synthetic.rb_ic(16, 12, seed=60 + s, amp=1.0))
        dX = imex.rk_tangent(p, stages, d, dt, *tab)
        assert abs(inner(g, d) - inner(p.kinetic_energy_grad(X[-1]), dX[-1])) <= 1e-12 * abs(inner(g, d))
        eps = 1e-5 * np.linalg.norm(X0) / np.linalg.norm(d)
        fd = (Jf(X0 + eps * d) - Jf(X0 - eps * d)) / (2 * eps)
        assert abs(fd - inner(g, d)) <= 1e-6 * abs(fd)
