"""3D plane Couette flow, Fourier(x, y) x Chebyshev(z) with tau terms (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Perturbation u = (u, v, w) of the laminar profile U(z) = z between walls at z = -1, +1
moving with velocities -1, +1, on x in [0, Lx), y in [0, Ly) (periodic):

    dt u - nu lap u + U dx u + w U' e_x + grad p = u x omega,   omega = curl u,
    div u = 0,   u = v = w = 0 at z = -1, +1,   int p dz = 0 on the mean pencil,

nu = 1/Re.  ``base="poiseuille"`` replaces the laminar profile by plane Poiseuille (channel) flow
U(z) = 1 - z^2 between stationary walls (U' = -2 z; the mean pressure gradient that drives it
stays fixed), the profile of the paper's Parametric sensitivity example; everything else is
unchanged.  The nonlinear term is written in rotational form, so p is the dynamic pressure
(pressure plus |u|^2/2); the terms linear in the perturbation (advection by U and the
shear production w U') are implicit.  IVP form M dX/dt + L X = F(X) (Supplementary A.4).

Every horizontal wavenumber pair (kx, ky) is an independent pencil (the paper's
"separable over wavenumbers" structure), discretised in z by the ultraspherical method
(Sparse spectral methods section) exactly as the Rayleigh-Benard pencils are:

* momentum rows are projected on C^(2), continuity on C^(1);
* the first-order tau reduction lifts tau_q1 onto the last C^(1) mode (entering the
  q-equation through d/dz of that mode, row N-2 of C^(2), and the continuity row N-1 for
  q = w) and tau_q2 onto the last C^(2) mode; tau_p (mean pencil only) enters continuity as
  a constant and pairs with the gauge int p dz = 0;
* the non-constant coefficient U(z) = z: the product z * u is formed exactly in the T basis
  (degree N, one more than u) and then converted with S1 S0 and truncated to the N C^(2)
  rows (Reading: the product is projected, not pre-truncated);
* nonlinear terms are evaluated on the 3/2-dealiased grid (Mx = 3Nx/2, My = 3Ny/2 Fourier
  points, Mz = 3Nz/2 Gauss points) and converted to C^(2) with S1 S0.

Pencil variable vector (length 4N + 7):
  [u_0..u_{N-1}, v_*, w_*, p_*, tau_u1, tau_u2, tau_v1, tau_v2, tau_w1, tau_w2, tau_p]
Equation rows:
  [u-eq (N), v-eq (N), w-eq (N), continuity (N), u(-1), u(1), v(-1), v(1), w(-1), w(1), gauge]

Storage: pencils [kx][ky] with kx = 0..Nx/2-1 (half spectrum, Nyquist not stored) and ky
index j = 0..Ny-1 in FFT order (ky = j or j - Ny); the ky = -Ny/2 row is held at zero and the
kx = 0 plane Hermitian (X(0, -ky) = conj X(0, ky)) by the orthogonal projection ``project``
applied after every solve.  Grid layout [x][y][z].
"""
import numpy as np
import scipy.linalg as sla

from . import chebyshev as cb
from . import fourier


class Couette:
    NTAU = 7

    def __init__(self, Nx, Ny, Nz, Re, Lx=4.0 * np.pi, Ly=2.0 * np.pi, dealias=1.5, nonlinear=True, pencils=True,
                 base="couette"):
        assert Nx % 2 == 0 and Ny % 2 == 0 and Nz >= 6 and base in ("couette", "poiseuille")
        self.base = base
        self.Nx, self.Ny, self.Nz = Nx, Ny, Nz
        self.Kx = Nx // 2
        self.Mx, self.My, self.Mz = (int(round(dealias * n)) for n in (Nx, Ny, Nz))
        self.Lx, self.Ly = float(Lx), float(Ly)
        self.Re = float(Re)
        self.nu = 1.0 / self.Re
        self.nonlinear = nonlinear
        N = self.N = Nz
        self.nvar = 4 * N + self.NTAU
        self.alpha = 2.0 * np.pi / self.Lx * np.arange(self.Kx)
        self.kyi = np.fft.fftfreq(Ny, 1.0 / Ny).astype(int)
        self.beta = 2.0 * np.pi / self.Ly * self.kyi
        self.SS = cb.S1(N) @ cb.S0(N)
        self.DD = cb.D1(N) @ cb.D0(N)
        self.SD = cb.S1(N) @ cb.D0(N)
        self.S0m, self.D0m = cb.S0(N), cb.D0(N)
        # z * T_n in the T basis of degree N (one extra row), then S1 S0 on N + 1 modes,
        # truncated to N rows: the C^(2) projection of the exact product.
        Zt = np.zeros((N + 1, N))
        Zt[1, 0] = 1.0
        for n in range(1, N):
            Zt[n + 1, n] += 0.5
            Zt[n - 1, n] += 0.5
        self.ZS = (cb.S1(N + 1) @ cb.S0(N + 1) @ Zt)[:N, :]
        if base == "couette":  # U = z, U' = 1
            self.Umat, self.UPmat = self.ZS, self.SS
        else:  # channel: U = 1 - z^2 (stationary walls), U' = -2 z; z^2 T_n exact in degree N + 1
            Zt2 = np.zeros((N + 2, N + 1))
            Zt2[1, 0] = 1.0
            for n in range(1, N + 1):
                Zt2[n + 1, n] += 0.5
                Zt2[n - 1, n] += 0.5
            one = np.zeros((N + 2, N))
            one[:N, :] = np.eye(N)
            self.Umat = (cb.S1(N + 2) @ cb.S0(N + 2) @ (one - Zt2 @ Zt))[:N, :]
            self.UPmat = -2.0 * self.ZS
        self.Dz = cb.deriv_T(N)
        self.Cz = cb.c2g_matrix(N, self.Mz)
        self.Gz = cb.g2c_matrix(N, self.Mz)
        self.G = cb.gram(N)  # int_{-1}^{1} T_m T_n dz
        self._lu = {}
        if not pencils:  # transforms, F and the objective only (large sizes)
            return
        shape = (self.Kx, Ny, self.nvar, self.nvar)
        self.Mmat = np.zeros(shape, dtype=np.complex128)
        self.Lmat = np.zeros(shape, dtype=np.complex128)
        for m in range(self.Kx):
            for j in range(Ny):
                self.Mmat[m, j], self.Lmat[m, j] = self.pencil_matrices(self.alpha[m], self.beta[j],
                                                                        mean=(m == 0 and j == 0))

    # ---- pencil operators ---------------------------------------------------------------
    def pencil_matrices(self, a, b, mean=False):
        """Dense (M, L) of the pencil with wavenumbers (kx, ky) = (a, b)."""
        N, nu = self.N, self.nu
        Mm = np.zeros((self.nvar, self.nvar), dtype=np.complex128)
        Lm = np.zeros((self.nvar, self.nvar), dtype=np.complex128)
        lift1 = -cb.D1(N)[:, N - 1]  # -(d/dz of the last C^(1) mode), in C^(2)
        bot, top = cb.boundary_rows(N)
        u, v, w, p = (slice(i * N, (i + 1) * N) for i in range(4))
        tu1, tu2, tv1, tv2, tw1, tw2, tp = range(4 * N, 4 * N + 7)
        lap = self.DD - (a * a + b * b) * self.SS
        adv = 1j * a * self.Umat  # U dx
        for blk in (u, v, w):
            Mm[blk, blk] = self.SS
            Lm[blk, blk] = -nu * lap + adv
        Lm[u, w] = self.UPmat  # w U' e_x
        Lm[u, p] = 1j * a * self.SS
        Lm[v, p] = 1j * b * self.SS
        Lm[w, p] = self.SD
        Lm[u, tu1] = nu * lift1
        Lm[v, tv1] = nu * lift1
        Lm[w, tw1] = nu * lift1
        Lm[N - 1, tu2] = 1.0
        Lm[2 * N - 1, tv2] = 1.0
        Lm[3 * N - 1, tw2] = 1.0
        Lm[p, u] = 1j * a * self.S0m  # continuity rows (C^(1))
        Lm[p, v] = 1j * b * self.S0m
        Lm[p, w] = self.D0m
        Lm[4 * N - 1, tw1] = 1.0
        r = 4 * N
        Lm[r + 0, u], Lm[r + 1, u] = bot, top
        Lm[r + 2, v], Lm[r + 3, v] = bot, top
        Lm[r + 4, w], Lm[r + 5, w] = bot, top
        if mean:
            Lm[3 * N, tp] = 1.0
            Lm[r + 6, p] = cb.integral_weights(N)
        else:
            Lm[r + 6, tp] = 1.0
        return Mm, Lm

    def eigenvalues(self, a, b):
        """Finite eigenvalues sigma of sigma M X + L X = 0 for the pencil (a, b) (linear
        stability of the laminar profile), sorted by decreasing real part."""
        Mm, Lm = self.pencil_matrices(a, b, mean=(a == 0 and b == 0))
        ev = sla.eig(-Lm, Mm, right=False)
        ev = ev[np.isfinite(ev)]
        return ev[np.argsort(-ev.real)]

    # ---- state <-> pencil vectors --------------------------------------------------------
    def pencils(self, state):
        """(3, Kx, Ny, N) velocity coefficients -> (Kx, Ny, nvar) (pressure, taus zero)."""
        X = np.zeros((self.Kx, self.Ny, self.nvar), dtype=np.complex128)
        for f in range(3):
            X[..., f * self.N:(f + 1) * self.N] = state[f]
        return X

    def state(self, X):
        N = self.N
        return np.stack([X[..., f * N:(f + 1) * N] for f in range(3)])

    def M(self, X):
        return np.einsum("abij,abj->abi", self.Mmat, X)

    def L(self, X):
        return np.einsum("abij,abj->abi", self.Lmat, X)

    def Mt(self, Y):
        return np.einsum("abji,abj->abi", self.Mmat.conj(), Y)

    def Lt(self, Y):
        return np.einsum("abji,abj->abi", self.Lmat.conj(), Y)

    def _factors(self, a, b):
        key = (float(a), float(b))
        if key not in self._lu:
            self._lu[key] = [[sla.lu_factor(a * self.Mmat[m, j] + b * self.Lmat[m, j]) for j in range(self.Ny)]
                             for m in range(self.Kx)]
        return self._lu[key]

    def solve(self, a, b, R):
        lu = self._factors(a, b)
        return np.array([[sla.lu_solve(lu[m][j], R[m, j]) for j in range(self.Ny)] for m in range(self.Kx)])

    def solve_t(self, a, b, R):
        lu = self._factors(a, b)
        return np.array([[sla.lu_solve(lu[m][j], R[m, j], trans=2) for j in range(self.Ny)]
                         for m in range(self.Kx)])

    def project(self, X):
        """Zero the ky = -Ny/2 row, make the kx = 0 plane Hermitian in ky (self-adjoint)."""
        X = np.array(X, dtype=np.complex128, copy=True)
        Ny = self.Ny
        X[:, Ny // 2] = 0.0
        neg = np.concatenate([[0], np.arange(Ny - 1, 0, -1)])
        X[0] = 0.5 * (X[0] + np.conj(X[0][neg]))
        X[0, Ny // 2] = 0.0
        return X

    # ---- 3D transforms of one field: coefficients (Kx, Ny, N) <-> grid (Mx, My, Mz) -------
    def _ypad(self, c):
        Ny, My = self.Ny, self.My
        out = np.zeros((c.shape[0], My) + c.shape[2:], dtype=np.complex128)
        out[:, :Ny // 2] = c[:, :Ny // 2]
        out[:, My - Ny // 2 + 1:] = c[:, Ny // 2 + 1:]
        return out

    def _ytrunc(self, c):
        Ny, My = self.Ny, self.My
        out = np.zeros((c.shape[0], Ny) + c.shape[2:], dtype=np.complex128)
        out[:, :Ny // 2] = c[:, :Ny // 2]
        out[:, Ny // 2 + 1:] = c[:, My - Ny // 2 + 1:]
        return out

    def c2g(self, c):
        m = c @ self.Cz.T                                          # z: (Kx, Ny, Mz)
        m = np.fft.ifft(self._ypad(m), axis=1) * self.My           # y: sum_ky c e^{i ky y}
        return fourier.c2g(m, self.Mx, axis=0)                     # x: real grid

    def g2c(self, g):
        m = fourier.g2c(g, self.Kx, axis=0)                        # x: (Kx, My, Mz)
        m = self._ytrunc(np.fft.fft(m, axis=1) / self.My)          # y
        return m @ self.Gz.T                                       # z

    def c2g_adj(self, g):
        m = fourier.c2g_adj(g, self.Kx, axis=0)
        m = self._ytrunc(np.fft.fft(m, axis=1))
        return m @ self.Cz

    def g2c_adj(self, c):
        m = c @ self.Gz
        m = np.fft.ifft(self._ypad(m), axis=1)
        return fourier.g2c_adj(m, self.Mx, axis=0)

    # ---- explicit term: u x omega --------------------------------------------------------
    def _ia(self):
        return 1j * self.alpha[:, None, None]

    def _ib(self):
        return 1j * self.beta[None, :, None]

    def fields(self, X):
        """Coefficients of (u, v, w, omega_x, omega_y, omega_z)."""
        u, v, w = self.state(X)
        dz = lambda c: c @ self.Dz.T
        ia, ib = self._ia(), self._ib()
        return [u, v, w, ib * w - dz(v), dz(u) - ia * w, ia * v - ib * u]

    def _grid(self, X):
        return [self.c2g(c) for c in self.fields(X)]

    def _embed(self, fx, fy, fz):
        Y = np.zeros((self.Kx, self.Ny, self.nvar), dtype=np.complex128)
        N = self.N
        for f, c in enumerate((fx, fy, fz)):
            Y[..., f * N:(f + 1) * N] = c @ self.SS.T
        return Y

    @staticmethod
    def _cross(g):
        u, v, w, ox, oy, oz = g
        return v * oz - w * oy, w * ox - u * oz, u * oy - v * ox

    def F(self, X):
        if not self.nonlinear:
            return np.zeros_like(X)
        return self._embed(*(self.g2c(f) for f in self._cross(self._grid(X))))

    def F_jvp(self, X, dX):
        if not self.nonlinear:
            return np.zeros_like(X)
        g, d = self._grid(X), self._grid(dX)
        u, v, w, ox, oy, oz = g
        du, dv, dw, dox, doy, doz = d
        fx = dv * oz + v * doz - dw * oy - w * doy
        fy = dw * ox + w * dox - du * oz - u * doz
        fz = du * oy + u * doy - dv * ox - v * dox
        return self._embed(self.g2c(fx), self.g2c(fy), self.g2c(fz))

    def F_vjp(self, X, Y):
        """Reverse sweep through F: embed^dagger ((S1 S0)^T), T^dagger, the cross product,
        (T^-1)^dagger and the adjoints of the vorticity multipliers ((i k)^dagger = -i k,
        Dz^dagger = Dz^T)."""
        if not self.nonlinear:
            return np.zeros_like(Y)
        N = self.N
        u, v, w, ox, oy, oz = self._grid(X)
        gx, gy, gz = (self.g2c_adj(Y[..., f * N:(f + 1) * N] @ self.SS) for f in range(3))
        bar = [
            -gy * oz + gz * oy,      # u
            gx * oz - gz * ox,       # v
            -gx * oy + gy * ox,      # w
            gy * w - gz * v,         # omega_x
            -gx * w + gz * u,        # omega_y
            gx * v - gy * u,         # omega_z
        ]
        cu, cv, cw, cox, coy, coz = (self.c2g_adj(b) for b in bar)
        ia, ib = self._ia(), self._ib()
        dzt = lambda c: c @ self.Dz
        out = np.zeros((self.Kx, self.Ny, self.nvar), dtype=np.complex128)
        out[..., 0:N] = cu + dzt(coy) + np.conj(-ib) * coz
        out[..., N:2 * N] = cv - dzt(cox) + np.conj(ia) * coz
        out[..., 2 * N:3 * N] = cw + np.conj(ib) * cox + np.conj(-ia) * coy
        return out

    # ---- objective: energy gain ----------------------------------------------------------
    # E(X) = (1/V) int |u|^2 dV = 1/2 sum_{kx, ky} w_kx sum_{u, v, w} c^H G c (Parseval over
    # the half spectrum in x, w_0 = 1, w_kx = 2; V = Lx Ly 2), the squared volume-weighted norm
    # of the paper's optimal-perturbation objective.  J = E(X_N) / E(X_0).
    def _wk(self):
        w = np.full(self.Kx, 2.0)
        w[0] = 1.0
        return w

    def energy(self, X):
        wk = self._wk()
        e = 0.0
        for c in self.state(X):
            e += 0.5 * float(np.sum(wk[:, None] * np.real(np.einsum("abi,ij,abj->ab", c.conj(), self.G, c))))
        return e

    def energy_grad(self, X):
        N = self.N
        wk = self._wk()
        out = np.zeros((self.Kx, self.Ny, self.nvar), dtype=np.complex128)
        for f, c in enumerate(self.state(X)):
            out[..., f * N:(f + 1) * N] = wk[:, None, None] * (c @ self.G.T)
        return out


def gain_gradient(prob, X0, nsteps, dt):
    """J = E(X_N) / E(X_0) and dJ/dX_0 by the multistep SBDF1 -> SBDF2 adjoint (store-all);
    the explicit dependence of J on X_0 enters at n = 0."""
    from . import imex
    X = imex.multistep_forward(prob, X0, nsteps, dt)
    E0, EN = prob.energy(X0), prob.energy(X[-1])
    J = EN / E0

    def dJ(n):
        if n == nsteps:
            g = prob.energy_grad(X[n]) / E0
            return g - (EN / E0 ** 2) * prob.energy_grad(X0) if n == 0 else g
        if n == 0:
            return -(EN / E0 ** 2) * prob.energy_grad(X0)
        return None

    g = imex.multistep_adjoint(prob, X, dJ, dt)
    return J, g, X


# ---- resolvent gains (linear operator of the pencils, energy norm) -------------------------
def resolvent_matrix(prob, a, b, omega):
    """R = prognostic part of (i omega M + L)^-1 [S1S0 f; 0] for the pencil (kx, ky) = (a, b):
    the response of (u, v, w) to a forcing f of the momentum equations at frequency omega
    (3N x 3N, T coefficients in and out)."""
    N = prob.N
    Mm, Lm = prob.pencil_matrices(a, b, mean=(a == 0 and b == 0))
    A = 1j * omega * Mm + Lm
    B = np.zeros((prob.nvar, 3 * N), dtype=np.complex128)
    for f in range(3):
        B[f * N:(f + 1) * N, f * N:(f + 1) * N] = prob.SS
    return np.linalg.solve(A, B)[:3 * N]


def resolvent_gain(prob, a, b, omega):
    """Leading gain sigma_1 = max ||R f||_E / ||f||_E in the energy norm ||c||_E^2 = c^H G3 c,
    G3 = blockdiag(G, G, G) (int T_m T_n dz), from the generalised Hermitian eigenproblem
    R^H G3 R f = sigma^2 G3 f."""
    import scipy.linalg as sla
    R = resolvent_matrix(prob, a, b, omega)
    G3 = sla.block_diag(prob.G, prob.G, prob.G)
    ev = sla.eigh(R.conj().T @ G3 @ R, G3, eigvals_only=True)
    return float(np.sqrt(ev[-1]))
