"""2D Kolmogorov flow in vorticity form on [0, 2 pi)^2 (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

    d_t w - (1/Re) lap w = -(u d_x w + v d_y w) - 4 cos(4y),
    u = d_y psi, v = -d_x psi, lap psi = -w,

the vorticity equation of the body force sin(4y) e_x.  IVP form M dX/dt + L X = F(X)
(Supplementary A.4) with M = I, L = |k|^2 / Re (diagonal), F evaluated pseudospectrally on
the 3/2-dealiased grid (Sparse spectral methods section), optionally plus a learned closure
term C(w; p) added on the grid (the CNN of ``oracle/cnn.py``), with p a parameter of F.

Coefficient layout per member: [kx][ky] complex with kx = 0..N/2-1 (half spectrum, Nyquist
not stored) and ky index j = 0..N-1 holding ky = j (j < N/2) or j - N (j >= N/2); the
ky = -N/2 row is held at zero and the kx = 0 column is held Hermitian (w(0, -ky) =
conj w(0, ky)) by the orthogonal projection ``project``, applied after every solve.
Grid layout [x_i][y_j], Mg = 3N/2 points per direction.
"""
import numpy as np

from . import fourier


class Kolmogorov:
    def __init__(self, N, Re, forcing=True, nonlinear=True, closure=None):
        assert N % 2 == 0
        self.N, self.Kx, self.Mg = N, N // 2, 3 * N // 2
        self.Re = float(Re)
        self.forcing, self.nonlinear, self.closure = forcing, nonlinear, closure
        kx = np.arange(self.Kx)
        ky = np.fft.fftfreq(N, 1.0 / N)  # 0..N/2-1, -N/2..-1
        self.kx = kx[:, None] * np.ones((1, N))
        self.ky = np.ones((self.Kx, 1)) * ky[None, :]
        self.k2 = self.kx ** 2 + self.ky ** 2
        self.inv_k2 = np.where(self.k2 > 0, 1.0 / np.where(self.k2 > 0, self.k2, 1.0), 0.0)
        self.nyq = (ky == -N // 2)
        self.fhat = np.zeros((self.Kx, N), dtype=np.complex128)
        if forcing:  # -4 cos(4y) = -2 e^{4iy} - 2 e^{-4iy}
            self.fhat[0, 4] = -2.0
            self.fhat[0, N - 4] = -2.0

    # ---- transforms (2D) -------------------------------------------------------------
    def _ypad(self, c):
        """[..., kx, ky(N)] -> [..., kx, M] zero-padded in natural FFT order."""
        N, M = self.N, self.Mg
        out = np.zeros(c.shape[:-1] + (M,), dtype=np.complex128)
        out[..., :N // 2] = c[..., :N // 2]
        out[..., M - N // 2 + 1:] = c[..., N // 2 + 1:]
        return out

    def _ytrunc(self, c):
        N, M = self.N, self.Mg
        out = np.zeros(c.shape[:-1] + (N,), dtype=np.complex128)
        out[..., :N // 2] = c[..., :N // 2]
        out[..., N // 2 + 1:] = c[..., M - N // 2 + 1:]
        return out

    def c2g(self, c):
        """B: coefficients [.., kx, ky] -> grid [.., x, y]."""
        W = np.fft.ifft(self._ypad(c), axis=-1) * self.Mg          # sum_ky c e^{i ky y}
        return fourier.c2g(W, self.Mg, axis=-2)

    def g2c(self, g):
        """T: grid -> coefficients (truncated)."""
        W = fourier.g2c(g, self.Kx, axis=-2)                       # (1/M) sum_x g e^{-i kx x}
        return self._ytrunc(np.fft.fft(W, axis=-1) / self.Mg)

    def c2g_adj(self, g):
        """B^dagger (factor 2 on kx >= 1 via the x adjoint; the y part is unitary up to M)."""
        W = fourier.c2g_adj(g, self.Kx, axis=-2)
        return self._ytrunc(np.fft.fft(W, axis=-1))

    def g2c_adj(self, c):
        """T^dagger."""
        W = np.fft.ifft(self._ypad(c), axis=-1)                    # (1/M) sum_ky c e^{i ky y}
        return fourier.g2c_adj(W, self.Mg, axis=-2)

    # ---- operators ----------------------------------------------------------------------
    def M_(self, X):
        return X

    def L(self, X):
        return self.k2 / self.Re * X

    def solve(self, a, b, R):
        return R / (a + b * self.k2 / self.Re)

    solve_t = solve
    Lt = L

    def project(self, X):
        X = np.array(X, dtype=np.complex128, copy=True)
        X[..., self.nyq] = 0.0
        col = X[..., 0, :]
        N = self.N
        neg = np.concatenate([[0], np.arange(N - 1, 0, -1)])  # index of -ky
        X[..., 0, :] = 0.5 * (col + np.conj(col[..., neg]))
        X[..., 0, N // 2] = 0.0
        return X

    def velocity_fields(self, X):
        psi = X * self.inv_k2
        u = 1j * self.ky * psi
        v = -1j * self.kx * psi
        wx = 1j * self.kx * X
        wy = 1j * self.ky * X
        return u, v, wx, wy

    def F(self, X):
        out = np.broadcast_to(self.fhat, X.shape).astype(np.complex128) if self.forcing else np.zeros_like(X)
        if self.nonlinear:
            u, v, wx, wy = (self.c2g(f) for f in self.velocity_fields(X))
            out = out - self.g2c(u * wx + v * wy)
        if self.closure is not None:
            out = out + self.g2c(self.closure.forward(self.c2g(X)))
        return out

    def F_jvp(self, X, dX):
        out = np.zeros_like(X)
        if self.nonlinear:
            u, v, wx, wy = (self.c2g(f) for f in self.velocity_fields(X))
            du, dv, dwx, dwy = (self.c2g(f) for f in self.velocity_fields(dX))
            out = out - self.g2c(du * wx + u * dwx + dv * wy + v * dwy)
        if self.closure is not None:
            out = out + self.g2c(self.closure.jvp(self.c2g(X), self.c2g(dX)))
        return out

    def F_vjp(self, X, Y):
        """(dF/dX)^dagger Y: T^dagger, the product rule, B^dagger and the adjoints of the
        spectral multipliers (i k)^dagger = -i k, (i k / |k|^2)^dagger = -i k / |k|^2."""
        out = np.zeros_like(Y)
        g = self.g2c_adj(Y)
        if self.nonlinear:
            u, v, wx, wy = (self.c2g(f) for f in self.velocity_fields(X))
            bu = self.c2g_adj(-g * wx)
            bv = self.c2g_adj(-g * wy)
            bwx = self.c2g_adj(-g * u)
            bwy = self.c2g_adj(-g * v)
            out = out + (-1j * self.ky * self.inv_k2) * bu + (1j * self.kx * self.inv_k2) * bv \
                + (-1j * self.kx) * bwx + (-1j * self.ky) * bwy
        if self.closure is not None:
            out = out + self.c2g_adj(self.closure.vjp(self.c2g(X), g))
        return out

    def F_param_vjp(self, X, Y):
        """(dF/dp)^dagger Y for the closure parameters (eq. 6: dJ/dp = -<Y, dF/dp>)."""
        return self.closure.param_vjp(self.c2g(X), self.g2c_adj(Y))

    # keep the generic names used by oracle.imex
    M = M_
    Mt = M_

    # ---- 4D-Var misfit ----------------------------------------------------------------
    def lowpass_mask(self, kmax=32):
        return ((np.abs(self.kx) <= kmax) & (np.abs(self.ky) <= kmax)).astype(np.float64)

    def misfit(self, X, obs, mask):
        d = mask * (X - obs)
        return 0.5 * float(np.sum(np.abs(d) ** 2))

    def misfit_grad(self, X, obs, mask):
        return mask * mask * (X - obs)


def fourdvar_gradient(prob, X0, nsteps, dt, obs_steps, obs, mask):
    """J = sum_m 1/2 ||H(w(t_m)) - obs_m||^2 and dJ/dX0 (multistep adjoint, cotangents
    injected at the observation steps)."""
    from . import imex
    X = imex.multistep_forward(prob, X0, nsteps, dt)
    J = sum(prob.misfit(X[n], obs[i], mask) for i, n in enumerate(obs_steps))
    idx = {n: i for i, n in enumerate(obs_steps)}
    dJ = lambda n: prob.misfit_grad(X[n], obs[idx[n]], mask) if n in idx else None
    g = imex.multistep_adjoint(prob, X, dJ, dt)
    return J, g, X
