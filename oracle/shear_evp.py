"""Linear stability eigenvalues of plane shear flows and their adjoint sensitivities (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eigenvalue problems (Problem types, "Eigenvalue problems"): the generalised problem

    (lambda M(p) + L(p)) X = 0,

its adjoint (conj(lambda) M^H + L^H) Y = 0, and the sensitivity of a simple eigenvalue to a
parameter p (eq. eigenvalue_sens, after Luchini & Bottaro 2014)

    dlambda/dp = - <Y, (lambda dM/dp + dL/dp) X> / <Y, M X>.

The flows are those of the Parametric sensitivity example and of the Couette problem: the
perturbation equations about a laminar profile U(z) e_x between walls at z = -1, +1,

    lambda u - nu lap u + U dx u + w U' e_x + grad p = 0,   div u = 0,   u = 0 at z = +-1,

nu = 1/Re, with U = 1 - z^2 (plane Poiseuille flow; the paper's y(2 - y) on [0, 2] written
in z = y - 1) or U = z (plane Couette flow).  A perturbation exp(i (alpha x + beta y)) is
one pencil; lambda = gamma + i omega with growth rate gamma = Re lambda.

The z discretisation is the Couette pencil's (same unknowns, equation rows and tau terms;
see ``oracle/couette.py``) with the base flow in place of z: U dx -> i alpha [U T_n] and
w U' e_x -> [U' T_n] in the u-row, the products U T_n and U' T_n formed exactly in the T
basis (degree N + 2 and N + 1), converted to C^(2) with S1 S0 and truncated to N rows.

The leading eigenpair comes from the dense QZ algorithm (scipy.linalg.eig with left and
right eigenvectors); the parameter derivatives of L are written out from the pencil's
definition.  ``neutral_re`` finds a point of the neutral curve gamma_max(Re, alpha) = 0 by
Newton's method in Re with dgamma/dRe from the sensitivity formula (the continuation step
of the Parametric sensitivity example).
"""
import numpy as np
import scipy.linalg as sla

from . import chebyshev as cb

BASE_FLOWS = ("couette", "poiseuille")


def _z_times(n_in):
    """(n_in + 1, n_in) matrix of multiplication by z in the Chebyshev-T basis:
    z T_0 = T_1, z T_n = (T_{n+1} + T_{n-1}) / 2."""
    Z = np.zeros((n_in + 1, n_in))
    Z[1, 0] = 1.0
    for n in range(1, n_in):
        Z[n + 1, n] += 0.5
        Z[n - 1, n] += 0.5
    return Z


class ShearEVP:
    """Pencil eigenproblem of plane Couette (U = z) or plane Poiseuille (U = 1 - z^2) flow with
    N Chebyshev modes per variable."""

    NTAU = 7

    def __init__(self, N, base="poiseuille"):
        assert base in BASE_FLOWS and N >= 6
        self.N, self.base = N, base
        self.nvar = 4 * N + self.NTAU
        self.SS = cb.S1(N) @ cb.S0(N)
        self.DD = cb.D1(N) @ cb.D0(N)
        self.SD = cb.S1(N) @ cb.D0(N)
        self.S0m, self.D0m = cb.S0(N), cb.D0(N)
        Z1 = _z_times(N)                      # z T_n, degree N
        Z2 = _z_times(N + 1) @ Z1             # z^2 T_n, degree N + 1
        conv = lambda B: (cb.S1(B.shape[0]) @ cb.S0(B.shape[0]) @ B)[:N, :]
        if base == "couette":
            self.Umat = conv(Z1)              # U = z
            self.UPmat = self.SS.copy()       # U' = 1
        else:
            one = np.zeros((N + 2, N))
            one[:N, :] = np.eye(N)
            self.Umat = conv(one - Z2)        # U = 1 - z^2
            self.UPmat = -2.0 * conv(Z1)      # U' = -2 z

    # ---- pencil ------------------------------------------------------------------------
    def matrices(self, a, b, Re):
        """Dense (M, L) of the pencil with wavenumbers (a, b) at Reynolds number Re."""
        N, nu = self.N, 1.0 / Re
        nv = self.nvar
        Mm = np.zeros((nv, nv), dtype=np.complex128)
        Lm = np.zeros((nv, nv), dtype=np.complex128)
        lift1 = -cb.D1(N)[:, N - 1]
        bot, top = cb.boundary_rows(N)
        u, v, w, p = (slice(i * N, (i + 1) * N) for i in range(4))
        tu1, tu2, tv1, tv2, tw1, tw2, tp = range(4 * N, 4 * N + 7)
        lap = self.DD - (a * a + b * b) * self.SS
        for blk in (u, v, w):
            Mm[blk, blk] = self.SS
            Lm[blk, blk] = -nu * lap + 1j * a * self.Umat
        Lm[u, w] = self.UPmat
        Lm[u, p] = 1j * a * self.SS
        Lm[v, p] = 1j * b * self.SS
        Lm[w, p] = self.SD
        Lm[u, tu1] = nu * lift1
        Lm[v, tv1] = nu * lift1
        Lm[w, tw1] = nu * lift1
        Lm[N - 1, tu2] = 1.0
        Lm[2 * N - 1, tv2] = 1.0
        Lm[3 * N - 1, tw2] = 1.0
        Lm[p, u] = 1j * a * self.S0m
        Lm[p, v] = 1j * b * self.S0m
        Lm[p, w] = self.D0m
        Lm[4 * N - 1, tw1] = 1.0
        r = 4 * N
        Lm[r + 0, u], Lm[r + 1, u] = bot, top
        Lm[r + 2, v], Lm[r + 3, v] = bot, top
        Lm[r + 4, w], Lm[r + 5, w] = bot, top
        if a == 0 and b == 0:
            Lm[3 * N, tp] = 1.0
            Lm[r + 6, p] = cb.integral_weights(N)
        else:
            Lm[r + 6, tp] = 1.0
        return Mm, Lm

    def dL(self, a, b, Re):
        """dL/dRe, dL/dalpha, dL/dbeta of the pencil (M does not depend on the parameters).
        Written out from ``matrices``: nu = 1/Re enters -nu lap and the tau lifts; alpha and
        beta enter lap, the advection i alpha U, the pressure gradient and continuity."""
        N, nu = self.N, 1.0 / Re
        nv = self.nvar
        dRe, da, db = (np.zeros((nv, nv), dtype=np.complex128) for _ in range(3))
        lift1 = -cb.D1(N)[:, N - 1]
        u, v, w, p = (slice(i * N, (i + 1) * N) for i in range(4))
        tu1, tv1, tw1 = 4 * N, 4 * N + 2, 4 * N + 4
        lap = self.DD - (a * a + b * b) * self.SS
        dnu = -1.0 / (Re * Re)
        for blk in (u, v, w):
            dRe[blk, blk] = -dnu * lap
            da[blk, blk] = 2.0 * a * nu * self.SS + 1j * self.Umat
            db[blk, blk] = 2.0 * b * nu * self.SS
        dRe[u, tu1] = dnu * lift1
        dRe[v, tv1] = dnu * lift1
        dRe[w, tw1] = dnu * lift1
        da[u, p] = 1j * self.SS
        db[v, p] = 1j * self.SS
        da[p, u] = 1j * self.S0m
        db[p, v] = 1j * self.S0m
        return dRe, da, db

    # ---- eigenpairs --------------------------------------------------------------------
    def eigs(self, a, b, Re):
        """All finite eigenvalues with right (X) and left (Y) eigenvectors, sorted by
        decreasing growth rate: -L X = lambda M X and Y^H (-L) = lambda Y^H M."""
        Mm, Lm = self.matrices(a, b, Re)
        lam, Y, X = sla.eig(-Lm, Mm, left=True, right=True)
        ok = np.isfinite(lam) & (np.abs(lam) < 1e8)
        lam, X, Y = lam[ok], X[:, ok], Y[:, ok]
        o = np.argsort(-lam.real)
        return lam[o], X[:, o], Y[:, o]

    def leading(self, a, b, Re, target=None):
        """The eigenpair of largest growth rate (or nearest ``target``): (lambda, X, Y)."""
        lam, X, Y = self.eigs(a, b, Re)
        i = 0 if target is None else int(np.argmin(np.abs(lam - target)))
        return lam[i], X[:, i], Y[:, i]

    def sensitivity(self, a, b, Re, lam, X, Y):
        """(dlambda/dRe, dlambda/dalpha, dlambda/dbeta) by eq. eigenvalue_sens."""
        Mm, _ = self.matrices(a, b, Re)
        den = np.vdot(Y, Mm @ X)
        return tuple(-np.vdot(Y, D @ X) / den for D in self.dL(a, b, Re))

    def neutral_re(self, a, Re0, b=0.0, tol=1e-13, max_iter=30):
        """Re on the neutral curve (gamma_max = 0) at wavenumber a by Newton's method in Re,
        dgamma/dRe = Re(dlambda/dRe) from the adjoint sensitivity.  Returns (Re, lambda,
        (dlambda/dRe, dlambda/dalpha, dlambda/dbeta))."""
        Re = float(Re0)
        for _ in range(max_iter):
            lam, X, Y = self.leading(a, b, Re)
            d = self.sensitivity(a, b, Re, lam, X, Y)
            step = lam.real / d[0].real
            Re -= step
            if abs(step) <= tol * Re:
                break
        lam, X, Y = self.leading(a, b, Re)
        return Re, lam, self.sensitivity(a, b, Re, lam, X, Y)

    # ---- prognostic (reduced) form used by shift-invert iterations ----------------------
    def shift_invert(self, a, b, Re, sigma):
        """Phi(sigma) = [(sigma M + L)^-1]_prog blockdiag(S1S0) (3N x 3N): the prognostic
        block of the shift-invert operator, whose eigenvalues are 1/(sigma - lambda)."""
        Mm, Lm = self.matrices(a, b, Re)
        N, H = self.N, 3 * self.N
        B = np.zeros((self.nvar, H), dtype=np.complex128)
        for f in range(3):
            B[f * N:(f + 1) * N, f * N:(f + 1) * N] = self.SS
        return sla.solve(sigma * Mm + Lm, B)[:H, :]
