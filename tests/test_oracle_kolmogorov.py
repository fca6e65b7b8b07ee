"""Pins for the Kolmogorov oracle (2D periodic vorticity, SBDF2, 4D-Var misfit).

* transforms: brute-force double sums (cos/sin) for a tiny size, trig polynomials exact,
  adjoint identities;
* F: brute-force evaluation by explicit sums; the laminar state w = -(Re/4) cos 4y is an
  exact fixed point of the discrete step; JVP = exact central difference; VJP = transpose
  of the brute-force Jacobian;
* linear modes follow the closed-form SBDF recurrence;
* 4D-Var gradient: dot test with the tangent, central FD, Taylor rate 2.
"""
import numpy as np
import pytest

import synthetic
from oracle import imex
from oracle import kolmogorov as ok
from oracle.imex import inner


def _herm(p, X):
    return p.project(X)


def brute_c2g(p, c):
    N, M = p.N, p.Mg
    xs = 2 * np.pi * np.arange(M) / M
    g = np.zeros((M, M))
    for a in range(p.Kx):
        for j in range(N):
            ky = p.ky[a, j]
            w = 1.0 if a == 0 else 2.0
            ph = np.exp(1j * (a * xs[:, None] + ky * xs[None, :]))
            g += w * np.real(c[a, j] * ph) if a > 0 else np.real(c[a, j] * ph)
    return g


def brute_g2c(p, g):
    N, M = p.N, p.Mg
    xs = 2 * np.pi * np.arange(M) / M
    c = np.zeros((p.Kx, N), complex)
    for a in range(p.Kx):
        for j in range(N):
            if p.nyq[j]:
                continue
            ky = p.ky[a, j]
            c[a, j] = np.sum(g * np.exp(-1j * (a * xs[:, None] + ky * xs[None, :]))) / M ** 2
    return c


def test_transforms_bruteforce_and_adjoints():
    p = ok.Kolmogorov(8, 100.0)
    rng = np.random.default_rng(0)
    c = _herm(p, rng.standard_normal((p.Kx, p.N)) + 1j * rng.standard_normal((p.Kx, p.N)))
    g = rng.standard_normal((p.Mg, p.Mg))
    np.testing.assert_allclose(p.c2g(c), brute_c2g(p, c), atol=1e-12)
    np.testing.assert_allclose(p.g2c(g), brute_g2c(p, g), atol=1e-13)
    np.testing.assert_allclose(p.g2c(p.c2g(c)), c, atol=1e-13)
    y = rng.standard_normal((p.Kx, p.N)) + 1j * rng.standard_normal((p.Kx, p.N))
    assert abs(inner(p.c2g(c), g) - inner(c, p.c2g_adj(g))) < 1e-11
    assert abs(inner(p.g2c(g), y) - inner(g, p.g2c_adj(y))) < 1e-12


def test_trig_polynomial_exact():
    p = ok.Kolmogorov(16, 100.0)
    xs = 2 * np.pi * np.arange(p.Mg) / p.Mg
    g = np.cos(3 * xs[:, None] + 2 * xs[None, :]) + 0.5 * np.sin(5 * xs[None, :])
    c = p.g2c(g)
    want = np.zeros((p.Kx, p.N), complex)
    want[3, 2] = 0.5
    want[0, 5] = 0.5 / (2j)
    want[0, p.N - 5] = -0.5 / (2j)
    np.testing.assert_allclose(c, want, atol=1e-15)


def test_F_bruteforce():
    p = ok.Kolmogorov(8, 100.0)
    rng = np.random.default_rng(1)
    X = _herm(p, rng.standard_normal((p.Kx, p.N)) + 1j * rng.standard_normal((p.Kx, p.N)))
    u, v, wx, wy = (brute_c2g(p, f) for f in p.velocity_fields(X))
    want = p.fhat - brute_g2c(p, u * wx + v * wy)
    np.testing.assert_allclose(p.F(X), want, atol=1e-12)


def test_laminar_fixed_point():
    N, Re, dt = 32, 100.0, 5e-3
    p = ok.Kolmogorov(N, Re)
    X = np.zeros((p.Kx, N), complex)
    X[0, 4] = X[0, N - 4] = -Re / 8.0       # w = -(Re/4) cos 4y
    np.testing.assert_allclose(p.F(X), p.fhat, atol=1e-12)
    Xs = imex.multistep_forward(p, X, 20, dt)
    np.testing.assert_allclose(Xs[-1], X, rtol=1e-13, atol=1e-12)


def test_linear_mode_recurrence():
    N, Re, dt, n = 16, 10.0, 1e-2, 30
    p = ok.Kolmogorov(N, Re, forcing=False, nonlinear=False)
    X0 = p.project(synthetic.kolmogorov_ic(N, 3))
    X = imex.multistep_forward(p, X0, n, dt)
    z = p.k2 / Re * dt
    x1 = X0 / (1 + z)
    disc = np.sqrt(4.0 - 2.0 * (1.5 + z) + 0j)
    r1, r2 = (2.0 + disc) / (2 * (1.5 + z)), (2.0 - disc) / (2 * (1.5 + z))
    B = (x1 - r1 * X0) / (r2 - r1)
    np.testing.assert_allclose(X[-1], (X0 - B) * r1 ** n + B * r2 ** n, rtol=1e-12, atol=1e-15)


def test_jvp_vjp():
    p = ok.Kolmogorov(8, 100.0)
    rng = np.random.default_rng(2)
    rand = lambda: _herm(p, rng.standard_normal((p.Kx, p.N)) + 1j * rng.standard_normal((p.Kx, p.N)))
    X = rand()
    d = rand()
    h = 1e-3
    fd = (p.F(X + h * d) - p.F(X - h * d)) / (2 * h)
    np.testing.assert_allclose(p.F_jvp(X, d), fd, atol=1e-11)
    n = p.Kx * p.N
    Jm = np.zeros((2 * n, 2 * n))
    for i in range(2 * n):
        e = np.zeros(2 * n)
        e[i] = 1.0
        Jm[:, i] = p.F_jvp(X, e.view(complex).reshape(p.Kx, p.N)).reshape(-1).view(float)
    for i in range(0, 2 * n, 5):
        e = np.zeros(2 * n)
        e[i] = 1.0
        v = p.F_vjp(X, e.view(complex).reshape(p.Kx, p.N)).reshape(-1).view(float)
        np.testing.assert_allclose(v, Jm[i], atol=1e-11)


@pytest.fixture(scope="module")
def fourdvar():
    N, Re, dt, nsteps = 32, 100.0, 5e-3, 40
    obs_steps = [10, 20, 30, 40]
    p = ok.Kolmogorov(N, Re)
    X0 = p.project(synthetic.kolmogorov_ic(N, 100))
    Xt = imex.multistep_forward(p, p.project(synthetic.kolmogorov_ic(N, 900)), nsteps, dt)
    mask = p.lowpass_mask(8)
    obs = np.stack([mask * Xt[n] for n in obs_steps])
    J, g, X = ok.fourdvar_gradient(p, X0, nsteps, dt, obs_steps, obs, mask)
    return p, X0, J, g, X, dt, nsteps, obs_steps, obs, mask


def test_fourdvar_dot_fd_taylor(fourdvar):
    p, X0, J, g, X, dt, nsteps, obs_steps, obs, mask = fourdvar
    # dot test: <g, d> = sum_m <dJ/dX_m, dX_m>
    d = p.project(synthetic.kolmogorov_ic(p.N, 7))
    dX = imex.multistep_tangent(p, X, d, dt)
    rhs = sum(inner(p.misfit_grad(X[n], obs[i], mask), dX[n]) for i, n in enumerate(obs_steps))
    assert abs(inner(g, d) - rhs) <= 1e-12 * abs(rhs)
    Jf = lambda Y0: ok.fourdvar_gradient(p, Y0, nsteps, dt, obs_steps, obs, mask)[0]
    for s in range(8):
        d = p.project(synthetic.kolmogorov_ic(p.N, 50 + s))
        eps = 1e-5 * np.linalg.norm(X0) / np.linalg.norm(d)
        fd = (Jf(X0 + eps * d) - Jf(X0 - eps * d)) / (2 * eps)
        assert abs(fd - inner(g, d)) <= 1e-6 * abs(fd)
    d = p.project(synthetic.kolmogorov_ic(p.N, 99))
    d *= 0.05 * np.linalg.norm(X0) / np.linalg.norm(d)
    rem = [abs(Jf(X0 + e * d) - J - e * inner(g, d)) for e in [0.4, 0.2, 0.1, 0.05]]
    rates = np.log2(np.array(rem[:-1]) / np.array(rem[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.05), rates


def test_ic_spectrum_and_rms():
    N = 64
    w = synthetic.kolmogorov_ic(N, 5)
    p = ok.Kolmogorov(N, 100.0)
    np.testing.assert_allclose(p.project(w), w, atol=1e-15)  # already admissible
    u, v, _, _ = p.velocity_fields(w)
    ug, vg = p.c2g(u), p.c2g(v)
    assert abs(np.mean(ug ** 2 + vg ** 2) - 1.0) < 1e-12
