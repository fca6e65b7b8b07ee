"""Pins for the plane-Couette oracle (Fourier x, y x Chebyshev tau in z, SBDF2).

* Transforms: brute-force double/triple sums on the grid; exact round trip; adjoint
  identities under the real inner product.
* Linear operator: the finite eigenvalues of every pencil reproduce those of an independent
  Chebyshev-collocation Orr-Sommerfeld + Squire solver (a different discretisation of the
  same linearised equations), which pins the pressure coupling, the advection U dx and the
  sign of the shear term w U'; the mean pencil decays at the Stokes rates -nu (n pi / 2)^2.
* Solver: the solution satisfies the no-slip conditions and continuity; transposed solve by
  the dot test.
* Nonlinear term u x omega: closed form for two analytic fields (streak and x-dependent
  roll); JVP = exact central difference (quadratic); VJP = transpose of the brute-force
  Jacobian.
* Objective: energy of an analytic field in closed form; the seeded initial field is
  divergence-free, vanishes at the walls and has the requested norm.
* Whole trajectory (SBDF1 -> SBDF2, energy gain): dot test between tangent and adjoint,
  central FD to 1e-6, Taylor rate 2; algebraic initial values inert.
"""
import numpy as np
import numpy.polynomial.chebyshev as C
import pytest
import scipy.linalg as sla

import synthetic
from oracle import couette as co
from oracle import imex
from oracle.imex import inner


def _rand_state(p, rng, hermitian=True):
    X = rng.standard_normal((p.Kx, p.Ny, p.nvar)) + 1j * rng.standard_normal((p.Kx, p.Ny, p.nvar))
    return p.project(X) if hermitian else X


def _field_values(p, c, x, y, z):
    """Brute-force value of the real field with coefficients c (Kx, Ny, N) at (x, y, z)."""
    Tn = np.cos(np.arange(p.N) * np.arccos(z))
    e = np.exp(1j * (p.alpha[:, None] * x + p.beta[None, :] * y))
    s = (c @ Tn) * e
    s[:, p.Ny // 2] = 0.0
    return float(np.real(s[0].sum()) + 2.0 * np.real(s[1:].sum()))


def test_transforms_bruteforce_and_adjoints():
    p = co.Couette(6, 4, 6, 100.0)
    rng = np.random.default_rng(0)
    c = p.state(_rand_state(p, rng))[0]
    g = p.c2g(c)
    xs = p.Lx * np.arange(p.Mx) / p.Mx
    ys = p.Ly * np.arange(p.My) / p.My
    zs = -np.cos(np.pi * (np.arange(p.Mz) + 0.5) / p.Mz)
    for i, j, k in [(0, 0, 0), (3, 2, 5), (8, 5, 1), (5, 1, 8)]:
        assert abs(g[i, j, k] - _field_values(p, c, xs[i], ys[j], zs[k])) < 1e-12
    np.testing.assert_allclose(p.g2c(g), c, atol=1e-13)
    # adjoints for arbitrary (not Hermitian-consistent) arguments
    cr = rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)
    gr = rng.standard_normal(g.shape)
    assert abs(np.sum(p.c2g(cr) * gr) - inner(cr, p.c2g_adj(gr))) < 1e-12 * np.sum(np.abs(gr))
    assert abs(inner(p.g2c(gr), cr) - np.sum(gr * p.g2c_adj(cr))) < 1e-12 * np.sum(np.abs(gr))


def _cheb(n):
    """Chebyshev-Gauss-Lobatto points and differentiation matrix (Trefethen, Spectral
    Methods in MATLAB, ch. 6)."""
    x = np.cos(np.pi * np.arange(n + 1) / n)
    c = np.ones(n + 1)
    c[0] = c[-1] = 2.0
    c *= (-1.0) ** np.arange(n + 1)
    X = np.tile(x[:, None], (1, n + 1))
    D = np.outer(c, 1.0 / c) / (X - X.T + np.eye(n + 1))
    return D - np.diag(D.sum(axis=1)), x


def _os_squire_eigs(a, b, Re, n=80):
    """Eigenvalues of the Orr-Sommerfeld (clamped, w = (1 - z^2) q) and Squire operators of
    U = z by collocation: sigma (D^2 - k^2) w = [nu (D^2 - k^2)^2 - i a U (D^2 - k^2)] w and
    sigma eta = [nu (D^2 - k^2) - i a U] eta."""
    D, x = _cheb(n)
    k2 = a * a + b * b
    D2 = D @ D
    S = np.diag(np.r_[0.0, 1.0 / (1.0 - x[1:-1] ** 2), 0.0])
    D4 = (np.diag(1 - x ** 2) @ np.linalg.matrix_power(D, 4) - 8 * np.diag(x) @ np.linalg.matrix_power(D, 3)
          - 12 * D2) @ S
    D2i, D4i, xi = D2[1:-1, 1:-1], D4[1:-1, 1:-1], x[1:-1]
    I = np.eye(n - 1)
    A = (D4i - 2 * k2 * D2i + k2 * k2 * I) / Re - 1j * a * np.diag(xi) @ (D2i - k2 * I)
    ev = np.concatenate([sla.eig(A, D2i - k2 * I, right=False),
                         np.linalg.eigvals((D2i - k2 * I) / Re - 1j * a * np.diag(xi))])
    return ev[np.isfinite(ev)]


@pytest.mark.parametrize("a,b", [(1.0, 1.0), (0.5, 2.0), (0.0, 1.0), (2.0, 0.0)])
def test_eigenvalues_match_orr_sommerfeld_squire(a, b):
    Re = 500.0
    p = co.Couette(4, 4, 48, Re)
    ours = p.eigenvalues(a, b)[:8]
    ref = _os_squire_eigs(a, b, Re)
    assert np.max(ref.real) < 0  # plane Couette is linearly stable
    for s in ours:
        assert np.min(np.abs(ref - s)) < 1e-6 * abs(s), (s, ref[np.argsort(np.abs(ref - s))[:2]])


def test_mean_pencil_stokes_decay():
    Re = 300.0
    p = co.Couette(4, 4, 32, Re)
    e = p.eigenvalues(0.0, 0.0)[:8]
    n = np.array([1, 1, 2, 2, 3, 3, 4, 4])
    np.testing.assert_allclose(e.real, -(n * np.pi / 2) ** 2 / Re, rtol=1e-10)
    assert np.max(np.abs(e.imag)) < 1e-12


def test_lift_up_closed_form():
    """The eigenvalues above cannot see the sign of the shear term (for U'' = 0 the two signs
    give similar operators), so pin it by the lift-up solution: for a streamwise-independent
    roll (kx = 0) with u0 = 0 and vanishing viscosity, w and v stay constant and
    du/dt = -w U' gives u(t) = -t w0 exactly; BDF schemes reproduce fields linear in t."""
    Re, dt, nsteps = 1e9, 0.05, 20
    p = co.Couette(4, 4, 12, Re, nonlinear=False)
    P = np.polynomial.Polynomial
    psi = P([1.0, 0.0, -1.0]) ** 2  # streamfunction cos(y) (1 - z^2)^2: v = dpsi/dz, w = -dpsi/dy
    s = np.zeros((3, p.Kx, p.Ny, p.N), complex)
    for j, ky in ((1, 1.0), (p.Ny - 1, -1.0)):
        s[1, 0, j] = 0.5 * _cheb_coeffs(psi.deriv(), p.N)
        s[2, 0, j] = -1j * ky * 0.5 * _cheb_coeffs(psi, p.N)
    X = imex.multistep_forward(p, p.pencils(s), nsteps, dt)
    u, v, w = p.state(X[-1])
    T = nsteps * dt
    scale = np.max(np.abs(s[2]))
    np.testing.assert_allclose(u, -T * s[2], atol=1e-6 * T * scale)
    np.testing.assert_allclose(v, s[1], atol=1e-6 * scale)
    np.testing.assert_allclose(w, s[2], atol=1e-6 * scale)


def test_solve_satisfies_constraints_and_transpose():
    p = co.Couette(8, 6, 16, 1000.0)
    N = p.N
    rng = np.random.default_rng(1)
    R = np.zeros((p.Kx, p.Ny, p.nvar), complex)
    R[..., :3 * N] = rng.standard_normal((p.Kx, p.Ny, 3 * N)) + 1j * rng.standard_normal((p.Kx, p.Ny, 3 * N))
    X = p.solve(1.5 / 5e-3, 1.0, R)
    scale = np.max(np.abs(X[..., :3 * N]))
    for f in range(3):
        c = X[..., f * N:(f + 1) * N]
        for zb in (-1.0, 1.0):
            assert np.max(np.abs(C.chebval(zb, np.moveaxis(c, -1, 0)))) < 1e-13 * scale
    u, v, w = p.state(X)
    div = (1j * p.alpha[:, None, None] * u + 1j * p.beta[None, :, None] * v) @ p.S0m.T + w @ p.D0m.T
    assert np.max(np.abs(div[..., :N - 1])) < 1e-10 * scale
    Y = rng.standard_normal(R.shape) + 1j * rng.standard_normal(R.shape)
    lhs = inner(Y, p.solve(1.5 / 5e-3, 1.0, R))
    rhs = inner(p.solve_t(1.5 / 5e-3, 1.0, Y), R)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def _cheb_coeffs(poly, N):
    c = C.poly2cheb(poly.coef)
    out = np.zeros(N)
    out[:len(c)] = c
    return out


def _closed_form_check(p, s, want):
    """F(X) for the state s against want(x, y, z) -> (Fx, Fy, Fz), at scattered points."""
    Fx = p.F(p.pencils(s))
    N = p.N
    for f in range(3):
        coef = np.linalg.solve(p.SS, np.moveaxis(Fx[..., f * N:(f + 1) * N], -1, 0).reshape(N, -1))
        coef = np.moveaxis(coef.reshape(N, p.Kx, p.Ny), 0, -1)
        for (x, y, z) in [(0.3, 1.1, -0.7), (2.9, 4.0, 0.2), (7.7, 5.5, 0.93), (11.0, 0.4, -0.05)]:
            assert abs(_field_values(p, coef, x, y, z) - want(x, y, z)[f]) < 1e-13


def test_F_closed_form_streak():
    # u = a(z) cos y with a = 1 - z^2:  u x omega = (0, -a^2 sin 2y / 2, a a' cos^2 y)
    p = co.Couette(16, 8, 12, 1000.0)
    P = np.polynomial.Polynomial
    a = P([1.0, 0.0, -1.0])
    s = np.zeros((3, p.Kx, p.Ny, p.N), complex)
    s[0, 0, 1] = s[0, 0, p.Ny - 1] = 0.5 * _cheb_coeffs(a, p.N)
    _closed_form_check(p, s, lambda x, y, z: (0.0, -a(z) ** 2 * np.sin(2 * y) / 2,
                                              a(z) * a.deriv()(z) * np.cos(y) ** 2))


def test_F_closed_form_roll():
    # v = b(z) cos x, w = c(z) sin x (x = 2 pi m / Lx with m = 2):
    # u x omega = ((c^2 - b^2) sin 2x / 2, -c b' sin 2x / 2, b b' cos^2 x)
    p = co.Couette(16, 8, 12, 1000.0)
    P = np.polynomial.Polynomial
    b = P([0.3, 1.0, -0.5, 0.2])
    cz = P([1.0, 0.0, -1.0]) * P([0.5, 1.0])
    s = np.zeros((3, p.Kx, p.Ny, p.N), complex)
    s[1, 2, 0] = 0.5 * _cheb_coeffs(b, p.N)
    s[2, 2, 0] = -0.5j * _cheb_coeffs(cz, p.N)
    _closed_form_check(p, s, lambda x, y, z: ((cz(z) ** 2 - b(z) ** 2) * np.sin(2 * x) / 2,
                                              -cz(z) * b.deriv()(z) * np.sin(2 * x) / 2,
                                              b(z) * b.deriv()(z) * np.cos(x) ** 2))


def test_F_jvp_vjp():
    p = co.Couette(4, 4, 6, 1000.0)
    rng = np.random.default_rng(5)
    X = _rand_state(p, rng)
    for _ in range(3):
        d = _rand_state(p, rng)
        h = 1e-3
        fd = (p.F(X + h * d) - p.F(X - h * d)) / (2 * h)
        np.testing.assert_allclose(p.F_jvp(X, d), fd, atol=1e-10 * np.max(np.abs(fd)))
    shape = (p.Kx, p.Ny, p.nvar)
    n = int(np.prod(shape))
    Jm = np.zeros((2 * n, 2 * n))
    for i in range(2 * n):
        e = np.zeros(2 * n)
        e[i] = 1.0
        Jm[:, i] = p.F_jvp(X, e.view(complex).reshape(shape)).reshape(-1).view(float)
    for i in range(0, 2 * n, 7):
        e = np.zeros(2 * n)
        e[i] = 1.0
        v = p.F_vjp(X, e.view(complex).reshape(shape)).reshape(-1).view(float)
        np.testing.assert_allclose(v, Jm[i], atol=1e-12 * np.max(np.abs(Jm)))


def test_energy_closed_form_and_ic():
    p = co.Couette(16, 8, 12, 1000.0)
    P = np.polynomial.Polynomial
    a = P([1.0, 0.0, -1.0])
    s = np.zeros((3, p.Kx, p.Ny, p.N), complex)
    s[0, 3, 2, :] = 0.5 * _cheb_coeffs(a, p.N)    # u = (1 - z^2) cos(3 x/2 + 2 y)
    # (1/V) int u^2 = 1/2 * 1/2 * int_{-1}^{1} (1 - z^2)^2 dz = 1/4 * 16/15
    assert abs(p.energy(p.pencils(s)) - 4.0 / 15.0) < 1e-14
    rng = np.random.default_rng(2)
    X = _rand_state(p, rng)
    d = _rand_state(p, rng)
    h = 1e-4
    fd = (p.energy(X + h * d) - p.energy(X - h * d)) / (2 * h)
    assert abs(fd - inner(p.energy_grad(X), d)) < 1e-10 * abs(fd)
    # seeded initial field: divergence-free, no-slip, norm 1e-4, Hermitian-consistent
    u0 = synthetic.couette_ic(16, 8, 12, seed=5)
    X0 = p.pencils(u0)
    assert abs(np.sqrt(p.energy(X0)) - 1e-4) < 1e-16
    np.testing.assert_allclose(p.project(X0), X0, atol=1e-20)
    u, v, w = u0
    div = 1j * p.alpha[:, None, None] * u + 1j * p.beta[None, :, None] * v + w @ p.Dz.T
    assert np.max(np.abs(div)) < 1e-18
    for c in u0:
        for zb in (-1.0, 1.0):
            assert np.max(np.abs(C.chebval(zb, np.moveaxis(c, -1, 0)))) < 1e-18


@pytest.fixture(scope="module")
def couette_traj():
    p = co.Couette(8, 6, 10, 300.0)
    X0 = p.pencils(synthetic.couette_ic(8, 6, 10, seed=5, norm=0.3))
    dt, nsteps = 2e-2, 25
    J, g, X = co.gain_gradient(p, X0, nsteps, dt)
    return p, X0, J, g, X, dt, nsteps


def test_couette_dot_test(couette_traj):
    p, X0, J, g, X, dt, nsteps = couette_traj
    rng = np.random.default_rng(7)
    for _ in range(2):
        d = _rand_state(p, rng)
        ybar = _rand_state(p, rng)
        dX = imex.multistep_tangent(p, X, d, dt)
        adj = imex.multistep_adjoint(p, X, lambda n: ybar if n == nsteps else None, dt)
        lhs, rhs = inner(adj, d), inner(ybar, dX[-1])
        assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_couette_gradient_fd_and_taylor(couette_traj):
    p, X0, J, g, X, dt, nsteps = couette_traj
    assert 0.0 < J < 10.0
    def Jf(X0_):
        return p.energy(imex.multistep_forward(p, X0_, nsteps, dt)[-1]) / p.energy(X0_)
    for s in range(6):
        d = p.pencils(synthetic.couette_ic(8, 6, 10, seed=100 + s, norm=1.0))
        if s % 2:
            d = d + _rand_state(p, np.random.default_rng(s)) * 0.1  # also off the divergence-free set
        eps = 1e-5 * np.linalg.norm(X0) / np.linalg.norm(d)
        fd = (Jf(X0 + eps * d) - Jf(X0 - eps * d)) / (2 * eps)
        assert abs(fd - inner(g, d)) <= 1e-6 * abs(fd)
    d = p.pencils(synthetic.couette_ic(8, 6, 10, seed=300, norm=1.0))
    d *= 0.3 * np.linalg.norm(X0) / np.linalg.norm(d)
    rem = []
    for e in [0.2, 0.1, 0.05, 0.025]:
        rem.append(abs(Jf(X0 + e * d) - J - e * inner(g, d)))
    rates = np.log2(np.array(rem[:-1]) / np.array(rem[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.1), rates


def test_couette_algebraic_initial_values_inert(couette_traj):
    p, X0, *_ = couette_traj
    Xb = X0.copy()
    Xb[..., 3 * p.N:] = 1.0 + 2.0j
    Xa = imex.multistep_forward(p, X0, 3, 2e-2)[-1]
    Xc = imex.multistep_forward(p, Xb, 3, 2e-2)[-1]
    np.testing.assert_array_equal(p.state(Xa), p.state(Xc))


def test_resolvent_gain_stokes_and_lift_up():
    """Resolvent gains in the energy norm.  Mean pencil: the operator is diffusion of u and v
    with no-slip walls, whose slowest mode decays at nu (pi/2)^2, so sigma_1 = 1/|i omega +
    nu (pi/2)^2|; the tau discretisation converges to it at fourth order in N.  Streamwise-
    independent pencil at omega = 0: lift-up makes sigma_1 grow as Re^2, sigma_1 / Re^2
    converging as Re grows."""
    for om in (0.0, 0.3):
        errs = []
        for N in (16, 24, 32):
            p = co.Couette(4, 4, N, 300.0, pencils=False)
            exact = 1.0 / np.hypot(om, p.nu * (np.pi / 2) ** 2)
            errs.append(abs(co.resolvent_gain(p, 0.0, 0.0, om) / exact - 1.0))
        rates = np.log(np.array(errs[:-1]) / np.array(errs[1:])) / np.log(np.array([24 / 16, 32 / 24]))
        assert errs[-1] < 1e-6 and np.all(rates > 3.5), (errs, rates)
    g = [co.resolvent_gain(co.Couette(4, 4, 48, Re, pencils=False), 0.0, 2.0, 0.0) / Re ** 2
         for Re in (1000.0, 2000.0, 4000.0)]
    d1, d2 = abs(g[1] / g[0] - 1), abs(g[2] / g[1] - 1)
    assert d1 < 2e-4 and 3.0 < d1 / d2 < 5.0, (g, d1, d2)  # sigma_1 = c Re^2 (1 + O(Re^-2))


def test_hessian_vector_product_fd_and_symmetry():
    """Tangent-over-adjoint Hessian-vector product of J = E(X_N): equals the central difference
    of the adjoint gradient (F is quadratic, so the FD error is O(eps^2)) and is symmetric."""
    p = co.Couette(8, 6, 10, 300.0)
    X0 = p.pencils(synthetic.couette_ic(8, 6, 10, seed=5, norm=0.3))
    n, dt = 12, 2e-2
    X = imex.multistep_forward(p, X0, n, dt)

    def grad(x0):
        Xs = imex.multistep_forward(p, x0, n, dt)
        return imex.multistep_adjoint(p, Xs, lambda k: p.energy_grad(Xs[k]) if k == n else None, dt)

    def hvp(v):
        dX = imex.multistep_tangent(p, X, v, dt)
        return imex.multistep_hvp(p, X, dX, lambda k: p.energy_grad(X[k]) if k == n else None,
                                  lambda k: p.energy_grad(dX[k]) if k == n else None, dt)

    v1 = p.pencils(synthetic.couette_ic(8, 6, 10, seed=77, norm=1.0))
    v2 = p.pencils(synthetic.couette_ic(8, 6, 10, seed=78, norm=1.0))
    h1, h2 = hvp(v1), hvp(v2)
    eps = 1e-4
    fd = (grad(X0 + eps * v1) - grad(X0 - eps * v1)) / (2 * eps)
    assert np.max(np.abs(h1 - fd)) <= 1e-8 * np.max(np.abs(fd))
    assert abs(inner(h1, v2) - inner(v1, h2)) <= 1e-12 * abs(inner(h1, v2))
