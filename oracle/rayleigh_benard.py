"""2D Rayleigh-Benard convection, Fourier(x) x Chebyshev(z) with tau terms (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Boussinesq equations in free-fall units on x in [0, Lx) (periodic), z in [0, 1], with
the buoyancy written as b = 1 - z + theta (conduction profile plus perturbation), so
all boundary conditions are homogeneous:

    dt u     - nu lap u + dx p         = -(u dx u + w dz u)
    dt w     - nu lap w + dz p - theta = -(u dx w + w dz w)
    dt theta - kappa lap theta - w     = -(u dx theta + w dz theta)
    dx u + dz w = 0,   u = w = theta = 0 at z = 0, 1,   int p = 0 (kx = 0 gauge)

with nu = (Ra/Pr)^(-1/2), kappa = (Ra Pr)^(-1/2).  IVP form M dX/dt + L X = F(X)
(Supplementary A.4).  Each x-wavenumber kx = 2 pi m / Lx (m = 0..Nx/2-1, Nyquist not
stored) is an independent pencil (the paper's "separable over wavenumbers" structure)
discretised by the ultraspherical method (Sparse spectral methods section):

* momentum and temperature rows are projected on C^(2), continuity on C^(1);
* tau terms (Lagrange multipliers for the boundary conditions) follow the first-order
  reduction grad q -> grad q + e_z lift(tau_q1) with lift onto the last C^(1) mode, so
  tau_q1 enters the q-equation through d/dz of that mode (row N-2 of C^(2)) and the
  continuity equation through tau_w1 (row N-1 of C^(1)); tau_q2 is lifted onto the last
  C^(2) mode; tau_p (kx = 0) enters continuity as a constant;
* nonlinear terms are evaluated on the 3/2-dealiased grid (Mx = 3Nx/2 Fourier points,
  Mz = 3Nz/2 Gauss points) and converted to C^(2) with S1 S0.

Variable vector per pencil (length 4N + 7):
  [u_0..u_{N-1}, w_*, theta_*, p_*, tau_u1, tau_u2, tau_w1, tau_w2, tau_t1, tau_t2, tau_p]
Equation rows per pencil:
  [u-eq (N), w-eq (N), theta-eq (N), continuity (N), u(0), u(1), w(0), w(1), t(0), t(1), gauge]
For kx != 0 the gauge row reads tau_p = 0 (tau_p only exists for the mean pencil).
The linear solves are dense LU factorisations of each pencil matrix a M + b L (cached
per (a, b): the paper reuses factorisations unless the timestep changes), and the
adjoint solves apply the Hermitian transpose of the same factors (Methods, "Linear
system solves").
"""
import numpy as np
import scipy.linalg as sla

from . import chebyshev as cb
from . import fourier


class RayleighBenard:
    NTAU = 7

    def __init__(self, Nx, Nz, Ra, Pr=1.0, Lx=4.0, dealias=1.5, nonlinear=True, x_sums="fft"):
        """x_sums = "direct" evaluates the x transforms as direct sums over explicit
        exponentials instead of numpy's FFT: the same maps, summed in another order (used to
        measure the rounding-order spread of long trajectories)."""
        assert Nx % 2 == 0 and Nz >= 4
        assert x_sums in ("fft", "direct")
        if x_sums == "fft":
            self._fx = (fourier.c2g, fourier.g2c, fourier.c2g_adj, fourier.g2c_adj)
        else:
            self._fx = (fourier.c2g_direct, fourier.g2c_direct, fourier.c2g_adj_direct, fourier.g2c_adj_direct)
        self.Nx, self.Nz = Nx, Nz
        self.Kx = Nx // 2
        self.Mx = int(round(dealias * Nx))
        self.Mz = int(round(dealias * Nz))
        self.Lx = float(Lx)
        self.Ra, self.Pr = float(Ra), float(Pr)
        self.nu = (Ra / Pr) ** -0.5
        self.kappa = (Ra * Pr) ** -0.5
        self.nonlinear = nonlinear
        self.kx = 2.0 * np.pi / self.Lx * np.arange(self.Kx)
        N = Nz
        self.N = N
        self.nvar = 4 * N + self.NTAU
        zs = 2.0  # d/dz = 2 d/dxi on z in [0, 1]
        self.SS = cb.S1(N) @ cb.S0(N)
        self.DD = cb.D1(N, zs) @ cb.D0(N, zs)
        self.SD = cb.S1(N) @ cb.D0(N, zs)
        self.S0m = cb.S0(N)
        self.D0m = cb.D0(N, zs)
        self.Dz = cb.deriv_T(N, zs)
        self.Cz = cb.c2g_matrix(N, self.Mz)
        self.Gz = cb.g2c_matrix(N, self.Mz)
        self.G = 0.5 * cb.gram(N)  # int_0^1 T_m T_n dz
        self.Mmat = np.zeros((self.Kx, self.nvar, self.nvar), dtype=np.complex128)
        self.Lmat = np.zeros((self.Kx, self.nvar, self.nvar), dtype=np.complex128)
        for m, k in enumerate(self.kx):
            self.Mmat[m], self.Lmat[m] = self.pencil_matrices(k, mean=(m == 0))
        self._lu = {}

    def pencil_matrices(self, k, mean=False):
        """Dense (M, L) of the pencil with x-wavenumber k (mean=True: the kx = 0 pencil)."""
        N, zs = self.N, 2.0
        Mm = np.zeros((self.nvar, self.nvar), dtype=np.complex128)
        Lm = np.zeros((self.nvar, self.nvar), dtype=np.complex128)
        lift1 = -cb.D1(N, zs)[:, N - 1]  # -(d/dz of the last C^(1) mode), in C^(2)
        bot, top = cb.boundary_rows(N)
        u, w, t, p = (slice(i * N, (i + 1) * N) for i in range(4))
        tu1, tu2, tw1, tw2, tt1, tt2, tp = range(4 * N, 4 * N + 7)
        lap = self.DD - k * k * self.SS
        for blk in (u, w, t):
            Mm[blk, blk] = self.SS
        Lm[u, u] = -self.nu * lap
        Lm[u, p] = 1j * k * self.SS
        Lm[u, tu1] = self.nu * lift1
        Lm[N - 1, tu2] = 1.0
        Lm[w, w] = -self.nu * lap
        Lm[w, p] = self.SD
        Lm[w, t] = -self.SS
        Lm[w, tw1] = self.nu * lift1
        Lm[2 * N - 1, tw2] = 1.0
        Lm[t, t] = -self.kappa * lap
        Lm[t, w] = -self.SS
        Lm[t, tt1] = self.kappa * lift1
        Lm[3 * N - 1, tt2] = 1.0
        Lm[p, u] = 1j * k * self.S0m     # continuity rows (C^(1))
        Lm[p, w] = self.D0m
        Lm[4 * N - 1, tw1] = 1.0
        r = 4 * N
        Lm[r + 0, u], Lm[r + 1, u] = bot, top
        Lm[r + 2, w], Lm[r + 3, w] = bot, top
        Lm[r + 4, t], Lm[r + 5, t] = bot, top
        if mean:
            Lm[3 * N, tp] = 1.0
            Lm[r + 6, p] = cb.integral_weights(N)
        else:
            Lm[r + 6, tp] = 1.0
        return Mm, Lm

    def growth_rate(self, k):
        """Largest real part of sigma with sigma M X + L X = 0 (linear stability of the
        conduction state at wavenumber k), from the dense generalised eigenproblem."""
        Mm, Lm = self.pencil_matrices(k)
        ev = sla.eig(-Lm, Mm, right=False)
        ev = ev[np.isfinite(ev)]
        return float(np.max(ev.real))

    # ---- state <-> pencil vectors ---------------------------------------------------
    def pencils(self, state):
        """(3, Kx, N) prognostic coefficients -> (Kx, nvar) pencil vectors (algebraic parts 0)."""
        X = np.zeros((self.Kx, self.nvar), dtype=np.complex128)
        for f in range(3):
            X[:, f * self.N:(f + 1) * self.N] = state[f]
        return X

    def state(self, X):
        N = self.N
        return np.stack([X[:, f * N:(f + 1) * N] for f in range(3)])

    # ---- linear operators (per pencil matrices) ----------------------------------------
    def M(self, X):
        return np.einsum("kij,kj->ki", self.Mmat, X)

    def L(self, X):
        return np.einsum("kij,kj->ki", self.Lmat, X)

    def Mt(self, Y):
        return np.einsum("kji,kj->ki", self.Mmat.conj(), Y)

    def Lt(self, Y):
        return np.einsum("kji,kj->ki", self.Lmat.conj(), Y)

    def _factors(self, a, b):
        key = (float(a), float(b))
        if key not in self._lu:
            self._lu[key] = [sla.lu_factor(a * self.Mmat[m] + b * self.Lmat[m]) for m in range(self.Kx)]
        return self._lu[key]

    def solve(self, a, b, R):
        lu = self._factors(a, b)
        return np.stack([sla.lu_solve(lu[m], R[m]) for m in range(self.Kx)])

    def solve_t(self, a, b, R):
        lu = self._factors(a, b)
        return np.stack([sla.lu_solve(lu[m], R[m], trans=2) for m in range(self.Kx)])

    def project(self, X):
        X = np.array(X, dtype=np.complex128, copy=True)
        X[0] = X[0].real
        return X

    # ---- 2D transforms of one field: coefficients (Kx, N) <-> grid (Mz, Mx) -----------------
    def c2g(self, c):
        return self._fx[0]((c @ self.Cz.T).T, self.Mx)

    def g2c(self, g):
        return self._fx[1](g, self.Kx).T @ self.Gz.T

    def c2g_adj(self, g):
        return self._fx[2](g, self.Kx).T @ self.Cz

    def g2c_adj(self, c):
        return self._fx[3]((c @ self.Gz).T, self.Mx)

    def dx(self, c):
        return 1j * self.kx[:, None] * c

    def dz(self, c):
        return c @ self.Dz.T

    # ---- explicit term ---------------------------------------------------------------
    def _grid_fields(self, X):
        u, w, t = self.state(X)
        return {"u": self.c2g(u), "w": self.c2g(w), "ux": self.c2g(self.dx(u)), "uz": self.c2g(self.dz(u)),
                "wx": self.c2g(self.dx(w)), "wz": self.c2g(self.dz(w)), "tx": self.c2g(self.dx(t)),
                "tz": self.c2g(self.dz(t))}

    def _embed(self, fu, fw, ft):
        Y = np.zeros((self.Kx, self.nvar), dtype=np.complex128)
        N = self.N
        Y[:, 0:N] = fu @ self.SS.T
        Y[:, N:2 * N] = fw @ self.SS.T
        Y[:, 2 * N:3 * N] = ft @ self.SS.T
        return Y

    def F(self, X):
        if not self.nonlinear:
            return np.zeros_like(X)
        g = self._grid_fields(X)
        fu = -(g["u"] * g["ux"] + g["w"] * g["uz"])
        fw = -(g["u"] * g["wx"] + g["w"] * g["wz"])
        ft = -(g["u"] * g["tx"] + g["w"] * g["tz"])
        return self._embed(self.g2c(fu), self.g2c(fw), self.g2c(ft))

    def F_jvp(self, X, dX):
        if not self.nonlinear:
            return np.zeros_like(X)
        g, d = self._grid_fields(X), self._grid_fields(dX)
        fu = -(d["u"] * g["ux"] + g["u"] * d["ux"] + d["w"] * g["uz"] + g["w"] * d["uz"])
        fw = -(d["u"] * g["wx"] + g["u"] * d["wx"] + d["w"] * g["wz"] + g["w"] * d["wz"])
        ft = -(d["u"] * g["tx"] + g["u"] * d["tx"] + d["w"] * g["tz"] + g["w"] * d["tz"])
        return self._embed(self.g2c(fu), self.g2c(fw), self.g2c(ft))

    def F_vjp(self, X, Y):
        """Reverse sweep through the evaluation of F: embed^dagger, (S1 S0)^T, T^dagger,
        the pointwise products, (T^-1)^dagger and the derivative adjoints (dx^dagger = -ik,
        dz^dagger = Dz^T)."""
        if not self.nonlinear:
            return np.zeros_like(Y)
        N = self.N
        g = self._grid_fields(X)
        cu = Y[:, 0:N] @ self.SS
        cw = Y[:, N:2 * N] @ self.SS
        ct = Y[:, 2 * N:3 * N] @ self.SS
        gu, gw, gt = self.g2c_adj(cu), self.g2c_adj(cw), self.g2c_adj(ct)
        bar = {
            "u": -(gu * g["ux"] + gw * g["wx"] + gt * g["tx"]),
            "w": -(gu * g["uz"] + gw * g["wz"] + gt * g["tz"]),
            "ux": -gu * g["u"], "uz": -gu * g["w"],
            "wx": -gw * g["u"], "wz": -gw * g["w"],
            "tx": -gt * g["u"], "tz": -gt * g["w"],
        }
        c = {k: self.c2g_adj(v) for k, v in bar.items()}
        dxa = lambda v: -1j * self.kx[:, None] * v
        dza = lambda v: v @ self.Dz
        out = np.zeros((self.Kx, self.nvar), dtype=np.complex128)
        out[:, 0:N] = c["u"] + dxa(c["ux"]) + dza(c["uz"])
        out[:, N:2 * N] = c["w"] + dxa(c["wx"]) + dza(c["wz"])
        out[:, 2 * N:3 * N] = dxa(c["tx"]) + dza(c["tz"])
        return out

    # ---- objective: kinetic energy at T ------------------------------------------------
    # J = 1/2 int int (u^2 + w^2) dz dx = (Lx/2) sum_{u,w} sum_k w_k c_k^H G c_k with
    # w_0 = 1, w_k = 2 (Parseval over the half spectrum) and G_mn = int_0^1 T_m T_n dz.
    def kinetic_energy(self, X):
        u, w, _ = self.state(X)
        e = 0.0
        for c in (u, w):
            e += float(np.real(c[0].conj() @ self.G @ c[0]))
            e += 2.0 * float(np.real(np.einsum("ki,ij,kj->", c[1:].conj(), self.G, c[1:])))
        return 0.5 * self.Lx * e

    def kinetic_energy_grad(self, X):
        N = self.N
        out = np.zeros((self.Kx, self.nvar), dtype=np.complex128)
        wk = np.full(self.Kx, 2.0)
        wk[0] = 1.0
        for f in (0, 1):
            c = X[:, f * N:(f + 1) * N].copy()
            c[0] = c[0].real
            out[:, f * N:(f + 1) * N] = self.Lx * wk[:, None] * (c @ self.G.T)
        return out

    def grid_points(self):
        x = self.Lx * np.arange(self.Mx) / self.Mx
        z = 0.5 * (cb.gauss_points(self.Mz) + 1.0)
        return x, z


def gradient(prob, X0, nsteps, dt, tableaux=None):
    """Kinetic energy at T and its gradient w.r.t. X_0 by the RK IMEX adjoint (store-all);
    ARS(2,2,2) unless other (A, H) tableaux are given."""
    from . import imex
    A, H = imex.rk222_tableaux() if tableaux is None else tableaux
    X, stages = imex.rk_forward(prob, X0, nsteps, dt, A, H)
    J = prob.kinetic_energy(X[-1])
    dJ = lambda n: prob.kinetic_energy_grad(X[n]) if n == nsteps else None
    g = imex.rk_adjoint(prob, stages, dJ, dt, A, H)
    return J, g, X, stages
