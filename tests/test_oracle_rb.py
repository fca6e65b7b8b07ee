"""Pins for the Rayleigh-Benard oracle (Fourier x Chebyshev tau, RK222).

* Discretisation: every pencil nonsingular (dense SVD at small N); the linear stability
  of the conduction state reproduces the textbook no-slip onset Ra_c = 1707.76 at
  k_c = 3.117 (growth rate changes sign across Ra_c at k_c, and is maximal near k_c).
* Solver: solution satisfies the boundary conditions and continuity; transposed solve
  by the dot test.
* RK222 (ARS(2,2,2)): closed-form amplification factor on linear diffusion, second-order
  convergence in dt (Supplementary A.4 RK stage equation).
* Nonlinear term: exact for analytic fields, JVP = exact central difference (quadratic),
  VJP = transpose of the brute-force Jacobian.
* Objective: kinetic energy of an analytic field in closed form.
* Whole trajectory: dot test between tangent and RK adjoint, central FD, Taylor rate 2;
  algebraic initial values do not change X_N.
"""
import numpy as np
import numpy.polynomial.chebyshev as C
import pytest

import synthetic
from oracle import burgers, imex
from oracle import rayleigh_benard as rb
from oracle.imex import inner


def test_pencils_nonsingular():
    p = rb.RayleighBenard(8, 8, 1e6)
    g = imex.RK222_GAMMA
    for m in range(p.Kx):
        s = np.linalg.svd(p.Mmat[m] + 1e-3 * g * p.Lmat[m], compute_uv=False)
        assert s.min() > 1e-12 * s.max()


def test_onset_constants():
    k_c, Ra_c = 3.117, 1707.76
    lo = rb.RayleighBenard(8, 24, Ra_c * 0.995)
    hi = rb.RayleighBenard(8, 24, Ra_c * 1.005)
    at = rb.RayleighBenard(8, 24, Ra_c)
    assert lo.growth_rate(k_c) < 0 < hi.growth_rate(k_c)
    assert abs(at.growth_rate(k_c)) < 5e-6
    assert at.growth_rate(k_c) > max(at.growth_rate(k_c - 0.15), at.growth_rate(k_c + 0.15))


def test_solve_satisfies_constraints_and_transpose():
    p = rb.RayleighBenard(8, 16, 1e6)
    N = p.N
    rng = np.random.default_rng(0)
    R = np.zeros((p.Kx, p.nvar), complex)
    R[:, :3 * N] = rng.standard_normal((p.Kx, 3 * N)) + 1j * rng.standard_normal((p.Kx, 3 * N))
    X = p.solve(1.0, 1e-3, R)
    scale = np.max(np.abs(X[:, :3 * N]))
    for f in range(3):
        c = X[:, f * N:(f + 1) * N]
        assert np.max(np.abs(C.chebval(-1.0, c.T))) < 1e-13 * scale
        assert np.max(np.abs(C.chebval(1.0, c.T))) < 1e-13 * scale
    u, w = X[:, :N], X[:, N:2 * N]
    div = p.dx(u) @ p.S0m.T + w @ p.D0m.T  # continuity in C^(1): modes 0..N-2 (last mode holds tau)
    assert np.max(np.abs(div[:, :N - 1])) < 1e-9 * np.max(np.abs(X[:, :3 * N]))
    Y = rng.standard_normal((p.Kx, p.nvar)) + 1j * rng.standard_normal((p.Kx, p.nvar))
    lhs = inner(Y, p.solve(1.0, 1e-3, R))
    rhs = inner(p.solve_t(1.0, 1e-3, Y), R)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_rk222_amplification_closed_form():
    N, nu, dt, nsteps = 16, 0.3, 1e-2, 40
    prob = burgers.Burgers(N, nu, nonlinear=False)
    X0 = synthetic.random_coeffs(N // 2, seed=8)
    X0[0] = X0[0].real
    A, H = imex.rk222_tableaux()
    X, _ = imex.rk_forward(prob, X0, nsteps, dt, A, H)
    g = imex.RK222_GAMMA
    z = nu * prob.k ** 2 * dt
    R = (1.0 - (1.0 - g) * z / (1.0 + g * z)) / (1.0 + g * z)
    np.testing.assert_allclose(X[-1], X0 * R ** nsteps, rtol=1e-13, atol=1e-16)


def test_rk222_second_order_cole_hopf():
    from tests.test_oracle_burgers import cole_hopf
    from oracle import fourier
    N, nu, eps, T = 64, 0.1, 0.8, 0.4
    prob = burgers.Burgers(N, nu)
    xg = prob.grid_points()
    X0 = fourier.g2c(cole_hopf(xg, 0.0, nu, eps), prob.K)
    A, H = imex.rk222_tableaux()
    errs = []
    for nsteps in [40, 80, 160]:
        X, _ = imex.rk_forward(prob, X0, nsteps, T / nsteps, A, H)
        errs.append(np.max(np.abs(prob.to_grid(X[-1]) - cole_hopf(xg, T, nu, eps))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.15), (errs, rates)


def _analytic_state(p):
    """u = cos(kx x) z(1-z), w = sin(kx x)(z - 1/2) z (1 - z) / 2, theta = cos(2 kx x) z^2 (1-z)."""
    N, Lx = p.N, p.Lx
    k1 = 2 * np.pi / Lx
    def cheb_of(poly):  # coefficients in T_n(xi), z = (xi+1)/2
        xi = np.polynomial.Polynomial([0.5, 0.5])
        c = C.poly2cheb(poly(xi).coef)
        out = np.zeros(N)
        out[:len(c)] = c
        return out
    Z = np.polynomial.Polynomial([0, 1])
    pu = Z * (1 - Z)
    pw = 0.5 * (Z - 0.5) * Z * (1 - Z)
    pt = Z * Z * (1 - Z)
    s = np.zeros((3, p.Kx, N), complex)
    s[0, 1] = 0.5 * cheb_of(pu)          # cos -> c_1 = 1/2
    s[1, 1] = -0.5j * cheb_of(pw)        # sin -> c_1 = 1/(2i)
    s[2, 2] = 0.5 * cheb_of(pt)
    fields = dict(u=lambda x, z: np.cos(k1 * x) * pu(z), w=lambda x, z: np.sin(k1 * x) * pw(z),
                  t=lambda x, z: np.cos(2 * k1 * x) * pt(z))
    d = dict(ux=lambda x, z: -k1 * np.sin(k1 * x) * pu(z), uz=lambda x, z: np.cos(k1 * x) * pu.deriv()(z),
             wx=lambda x, z: k1 * np.cos(k1 * x) * pw(z), wz=lambda x, z: np.sin(k1 * x) * pw.deriv()(z),
             tx=lambda x, z: -2 * k1 * np.sin(2 * k1 * x) * pt(z), tz=lambda x, z: np.cos(2 * k1 * x) * pt.deriv()(z))
    fields.update(d)
    return s, fields


def test_F_exact_for_analytic_fields():
    p = rb.RayleighBenard(16, 12, 1e6)
    s, f = _analytic_state(p)
    X = p.pencils(s)
    Fx = p.F(X)
    # back out the T coefficients of F from the C^(2) rows and evaluate them at arbitrary points
    N = p.N
    xs = np.array([0.13, 1.7, 3.1])
    zs = np.array([0.07, 0.5, 0.93])
    for row, (a, b) in zip(range(3), [("ux", "uz"), ("wx", "wz"), ("tx", "tz")]):
        coef = np.linalg.solve(p.SS, Fx[:, row * N:(row + 1) * N].T).T  # (Kx, N)
        for x in xs:
            for z in zs:
                xi = 2 * z - 1
                val = coef[0, :] @ np.cos(np.arange(N) * np.arccos(xi))
                val = val.real + 2 * np.real(np.sum(coef[1:] @ np.cos(np.arange(N) * np.arccos(xi))
                                                    * np.exp(1j * p.kx[1:] * x)))
                want = -(f["u"](x, z) * f[a](x, z) + f["w"](x, z) * f[b](x, z))
                assert abs(val - want) < 1e-13


def test_F_jvp_vjp():
    p = rb.RayleighBenard(4, 6, 1e6)
    rng = np.random.default_rng(5)
    def rand():
        X = rng.standard_normal((p.Kx, p.nvar)) + 1j * rng.standard_normal((p.Kx, p.nvar))
        return p.project(X)
    X = rand()
    for _ in range(3):
        d = rand()
        h = 1e-3
        fd = (p.F(X + h * d) - p.F(X - h * d)) / (2 * h)
        np.testing.assert_allclose(p.F_jvp(X, d), fd, atol=1e-10 * np.max(np.abs(fd)))
    n = p.Kx * p.nvar
    Jm = np.zeros((2 * n, 2 * n))
    for i in range(2 * n):
        e = np.zeros(2 * n)
        e[i] = 1.0
        Jm[:, i] = p.F_jvp(X, e.view(complex).reshape(p.Kx, p.nvar)).reshape(-1).view(float)
    for i in range(0, 2 * n, 3):
        e = np.zeros(2 * n)
        e[i] = 1.0
        v = p.F_vjp(X, e.view(complex).reshape(p.Kx, p.nvar)).reshape(-1).view(float)
        np.testing.assert_allclose(v, Jm[i], atol=1e-12 * np.max(np.abs(Jm)))


def test_kinetic_energy_closed_form():
    p = rb.RayleighBenard(16, 12, 1e6)
    N = p.N
    Z = np.polynomial.Polynomial([0, 1])
    xi = np.polynomial.Polynomial([0.5, 0.5])
    c = C.poly2cheb((Z * (1 - Z))(xi).coef)
    s = np.zeros((3, p.Kx, N), complex)
    s[0, 3, :len(c)] = 0.5 * c   # u = cos(3 k1 x) z (1-z)
    X = p.pencils(s)
    assert abs(p.kinetic_energy(X) - p.Lx / 120.0) < 1e-14
    # gradient of J by central differences along random directions
    rng = np.random.default_rng(1)
    d = p.project(rng.standard_normal((p.Kx, p.nvar)) + 1j * rng.standard_normal((p.Kx, p.nvar)))
    h = 1e-4
    fd = (p.kinetic_energy(X + h * d) - p.kinetic_energy(X - h * d)) / (2 * h)
    assert abs(fd - inner(p.kinetic_energy_grad(X), d)) < 1e-10 * abs(fd)


def rb_ic(p, seed=2, amp=1e-3):
    return p.pencils(synthetic.rb_ic(p.Nx, p.Nz, seed=seed, amp=amp))


@pytest.fixture(scope="module")
def rb_traj():
    p = rb.RayleighBenard(16, 12, 1e6)
    X0 = rb_ic(p, amp=0.3)
    dt, nsteps = 1e-2, 30
    J, g, X, stages = rb.gradient(p, X0, nsteps, dt)
    return p, X0, J, g, X, stages, dt, nsteps


def test_rb_dot_test(rb_traj):
    p, X0, J, g, X, stages, dt, nsteps = rb_traj
    A, H = imex.rk222_tableaux()
    for s in range(2):
        d = rb_ic(p, seed=50 + s, amp=1.0)
        dX = imex.rk_tangent(p, stages, d, dt, A, H)
        lhs = inner(g, d)
        rhs = inner(p.kinetic_energy_grad(X[-1]), dX[-1])
        assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_rb_gradient_fd_and_taylor(rb_traj):
    p, X0, J, g, X, stages, dt, nsteps = rb_traj
    A, H = imex.rk222_tableaux()
    Jf = lambda X0_: p.kinetic_energy(imex.rk_forward(p, X0_, nsteps, dt, A, H)[0][-1])
    for s in range(8):
        d = rb_ic(p, seed=100 + s, amp=1.0)
        eps = 1e-5 * np.linalg.norm(X0) / np.linalg.norm(d)
        fd = (Jf(X0 + eps * d) - Jf(X0 - eps * d)) / (2 * eps)
        assert abs(fd - inner(g, d)) <= 1e-6 * abs(fd)
    d = rb_ic(p, seed=300, amp=1.0)
    d *= 0.3 * np.linalg.norm(X0) / np.linalg.norm(d)
    rem = []
    for e in [0.2, 0.1, 0.05, 0.025]:
        rem.append(abs(Jf(X0 + e * d) - J - e * inner(g, d)))
    rates = np.log2(np.array(rem[:-1]) / np.array(rem[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.05), rates


def test_rb_algebraic_initial_values_inert(rb_traj):
    p, X0, *_ = rb_traj
    A, H = imex.rk222_tableaux()
    Xb = X0.copy()
    Xb[:, 3 * p.N:] = 1.0 + 2.0j
    Xa = imex.rk_forward(p, X0, 3, 1e-2, A, H)[0][-1]
    Xc = imex.rk_forward(p, Xb, 3, 1e-2, A, H)[0][-1]
    np.testing.assert_array_equal(p.state(Xa), p.state(Xc))
