"""1D viscous Burgers on a periodic Fourier basis (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

IVP in the paper's form M dX/dt + L X = F(X) (Supplementary A.4) with
M = I, L = nu k^2 (diagonal) and the conservative nonlinearity
F(u) = -d/dx (u^2 / 2), evaluated pseudospectrally on a 3/2-dealiased grid
(Sparse spectral methods section: nonlinear terms on a collocation grid via
fast transforms; Supplementary B: 3/2 dealiasing).

State: K = N/2 complex half-spectrum coefficients per batch member
(Nyquist not stored, Im c_0 held at zero by ``project``).
"""
import numpy as np

from . import fourier


class Burgers:
    def __init__(self, N, nu, length=2.0 * np.pi, dealias=1.5, nonlinear=True):
        assert N % 2 == 0
        self.N, self.K = N, N // 2
        self.Mg = int(round(dealias * N))
        self.nu = float(nu)
        self.length = float(length)
        self.k = 2.0 * np.pi / self.length * np.arange(self.K)
        self.nonlinear = nonlinear

    # grid helpers ------------------------------------------------------------------
    def to_grid(self, X):
        return fourier.c2g(X, self.Mg)

    def grid_points(self):
        return self.length * np.arange(self.Mg) / self.Mg

    # linear operators ------------------------------------------------------------------
    def M(self, X):
        return X

    Mt = M

    def L(self, X):
        return self.nu * self.k ** 2 * X

    Lt = L

    def solve(self, a, b, R):
        return R / (a + b * self.nu * self.k ** 2)

    solve_t = solve

    def project(self, X):
        X = np.array(X, dtype=np.complex128, copy=True)
        X[..., 0] = X[..., 0].real
        return X

    # explicit term -------------------------------------------------------------------
    def F(self, X):
        if not self.nonlinear:
            return np.zeros_like(X)
        u = fourier.c2g(X, self.Mg)
        return -1j * self.k * fourier.g2c(0.5 * u * u, self.K)

    def F_jvp(self, X, dX):
        if not self.nonlinear:
            return np.zeros_like(X)
        u = fourier.c2g(X, self.Mg)
        du = fourier.c2g(dX, self.Mg)
        return -1j * self.k * fourier.g2c(u * du, self.K)

    def F_vjp(self, X, Y):
        """(dF/dX)^dagger Y = B^dagger[ (B X) * T^dagger( (-i k)^dagger Y ) ], (-ik)^dagger = +ik."""
        if not self.nonlinear:
            return np.zeros_like(Y)
        u = fourier.c2g(X, self.Mg)
        gY = fourier.g2c_adj(1j * self.k * Y, self.Mg)
        return fourier.c2g_adj(u * gY, self.K)

    # objective J = 1/2 int u(T)^2 dx (physical L2 integral, by Parseval) --------------
    def energy(self, X):
        X = np.asarray(X)
        e = X[..., 0].real ** 2 + 2.0 * np.sum(np.abs(X[..., 1:]) ** 2, axis=-1)
        return 0.5 * self.length * e

    def energy_grad(self, X):
        g = 2.0 * self.length * np.asarray(X, dtype=np.complex128)
        g[..., 0] = self.length * X[..., 0].real
        return g


def gradient(prob, X0, nsteps, dt, order=2):
    """J = 1/2 ||u(T)||^2 and dJ/dX_0 by the multistep adjoint (store-all trajectory)."""
    from . import imex
    X = imex.multistep_forward(prob, X0, nsteps, dt, order)
    J = prob.energy(X[-1])
    dJ = lambda n: prob.energy_grad(X[n]) if n == nsteps else None
    g = imex.multistep_adjoint(prob, X, dJ, dt, order)
    return J, g, X
