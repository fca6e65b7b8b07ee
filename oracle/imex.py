"""IMEX timesteppers, their tangents and their exact discrete adjoints (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Notation follows Supplementary A.4 of arXiv 2506.14792: the IVP is
``M dX/dt + L X = F(X)``.  A problem object supplies, on complex coefficient
vectors (the real inner product is ``<a, b> = Re sum conj(a) b``):

* ``M(X)``, ``L(X)``, ``F(X)``            -- maps from variable space to equation space
* ``Mt(Y)``, ``Lt(Y)``                    -- their adjoints (equation -> variable space)
* ``F_jvp(X, dX)``, ``F_vjp(X, Y)``       -- Jacobian-vector / vector-Jacobian products of F
* ``solve(a, b, R)``                      -- X with (a M + b L) X = R
* ``solve_t(a, b, R)``                    -- Y with (a M + b L)^dagger Y = R
* ``project(X)``                          -- orthogonal projection onto the admissible
                                             (Hermitian-consistent) coefficients, applied
                                             after every solve; it is self-adjoint.

Scheme constants are the published methods the paper cites for its
timesteppers (Wang & Ruuth 2008 SBDF; Ascher, Ruuth & Spiteri 1997 ARS(2,2,2)).
"""
import math

import numpy as np


def inner(a, b):
    """Real inner product over the stored real numbers of two coefficient vectors."""
    return float(np.real(np.vdot(a, b)))


# --------------------------------------------------------------------------------------
# Scheme constants
# --------------------------------------------------------------------------------------

def sbdf_coeffs(n, order, dt):
    """Coefficients (a[0..s], b[0..s], c[0..s]) of step n (n >= 1) of SBDF<order>.

    Eq. imex: (a0 M + b0 L) X_n = sum_{i=1..s} [c_i F(X_{n-i}) - (a_i M + b_i L) X_{n-i}].
    The scheme falls back to a lower order while fewer than ``order`` past steps
    exist (the paper: "revert to lower order multistep IMEX schemes for early
    iterations").  c[0] is unused and set to 0.

    dt is a scalar (constant step) or a sequence of step sizes (step n spans dt[n-1]); with a
    sequence the weights come from the scheme's definition on the actual nodes
    t_n, t_{n-1}, ..., t_{n-s} (sbdf_weights_nodes): variable-step SBDF, which the paper's
    timesteppers need when the timestep changes (Supplementary A.4).
    """
    if np.ndim(dt):
        s = min(n, order)
        h = [float(dt[n - 1 - i]) for i in range(s)]  # h_n, h_{n-1}, ...: t_{n-i} - t_{n-i-1}
        nodes = [0.0]
        for i in range(s):
            nodes.append(nodes[-1] - h[i])
        a, c = sbdf_weights_nodes(nodes)
        b = np.zeros(s + 1)
        b[0] = 1.0
        return np.array(a), b, np.array(c)
    s = min(n, order)
    if s == 1:  # backward/forward Euler
        return (np.array([1.0 / dt, -1.0 / dt]), np.array([1.0, 0.0]), np.array([0.0, 1.0]))
    if s == 2:  # SBDF2 with constant dt
        return (np.array([1.5 / dt, -2.0 / dt, 0.5 / dt]), np.array([1.0, 0.0, 0.0]),
                np.array([0.0, 2.0, -1.0]))
    if s in (3, 4):
        a, c = sbdf_weights(s)
        b = np.zeros(s + 1)
        b[0] = 1.0
        return (np.array([float(v) for v in a]) / dt, b, np.array([float(v) for v in c]))
    raise ValueError("SBDF orders 1..4 are defined here")


def sbdf_weights(s):
    """Exact rational weights of SBDF<s> with constant step, from the scheme's definition: the
    implicit part is the backward differentiation formula, a_i = d/dt of the Lagrange basis
    polynomial of node t_{n-i} through the nodes t_n, ..., t_{n-s}, evaluated at t_n (times dt);
    the explicit part extrapolates F to t_n, c_i = the Lagrange basis polynomial of t_{n-i}
    through t_{n-1}, ..., t_{n-s}, evaluated at t_n (c_0 = 0).  Nodes in units of dt."""
    from fractions import Fraction as Fr
    nodes = [Fr(-i) for i in range(s + 1)]  # t_{n-i} - t_n
    a = []
    for i in range(s + 1):
        others = [nodes[j] for j in range(s + 1) if j != i]
        den = Fr(1)
        for o in others:
            den *= nodes[i] - o
        # derivative at 0 of prod (t - o): sum over o of prod over the rest of (0 - o')
        num = Fr(0)
        for k in range(len(others)):
            term = Fr(1)
            for m, o in enumerate(others):
                if m != k:
                    term *= -o
            num += term
        a.append(num / den)
    c = [Fr(0)]
    for i in range(1, s + 1):
        v = Fr(1)
        for j in range(1, s + 1):
            if j != i:
                v *= (0 - nodes[j]) / (nodes[i] - nodes[j])
        c.append(v)
    return a, c


def sbdf_weights_nodes(nodes):
    """SBDF weights from the scheme's definition on arbitrary nodes: nodes[i] = t_{n-i} - t_n
    (nodes[0] = 0, decreasing).  a_i = d/dt at t_n of the Lagrange basis polynomial of t_{n-i}
    through all the nodes (backward differentiation, in units of 1/time); c_i (i >= 1) = the
    Lagrange basis polynomial of t_{n-i} through t_{n-1}, ..., t_{n-s}, evaluated at t_n
    (extrapolation of F); c_0 = 0.  Floats in, floats out (sbdf_weights is the rational,
    constant-step form)."""
    s = len(nodes) - 1
    a = []
    for i in range(s + 1):
        others = [nodes[j] for j in range(s + 1) if j != i]
        den = 1.0
        for o in others:
            den *= nodes[i] - o
        num = 0.0
        for k in range(len(others)):
            term = 1.0
            for m, o in enumerate(others):
                if m != k:
                    term *= -o
            num += term
        a.append(num / den)
    c = [0.0]
    for i in range(1, s + 1):
        v = 1.0
        for j in range(1, s + 1):
            if j != i:
                v *= (0.0 - nodes[j]) / (nodes[i] - nodes[j])
        c.append(v)
    return a, c


RK222_GAMMA = 1.0 - 1.0 / math.sqrt(2.0)
RK222_DELTA = 1.0 - 1.0 / (2.0 * RK222_GAMMA)


def rk222_tableaux():
    """ARS(2,2,2): explicit tableau A[i][j] and implicit tableau H[i][j] (i, j = 0..2)."""
    g, d = RK222_GAMMA, RK222_DELTA
    A = np.array([[0.0, 0.0, 0.0], [g, 0.0, 0.0], [d, 1.0 - d, 0.0]])
    H = np.array([[0.0, 0.0, 0.0], [0.0, g, 0.0], [0.0, 1.0 - g, g]])
    return A, H


def rk443_tableaux():
    """ARS(4,4,3) (Ascher, Ruuth & Spiteri 1997, the Runge-Kutta IMEX family the paper's
    timesteppers follow): explicit tableau A[i][j] and implicit tableau H[i][j] (i, j = 0..4),
    third order, diagonal 1/2 on every implicit stage and a zero first implicit column."""
    A = np.zeros((5, 5))
    H = np.zeros((5, 5))
    A[1, 0] = 1.0 / 2.0
    A[2, 0], A[2, 1] = 11.0 / 18.0, 1.0 / 18.0
    A[3, 0], A[3, 1], A[3, 2] = 5.0 / 6.0, -5.0 / 6.0, 1.0 / 2.0
    A[4, 0], A[4, 1], A[4, 2], A[4, 3] = 1.0 / 4.0, 7.0 / 4.0, 3.0 / 4.0, -7.0 / 4.0
    H[1, 1] = 1.0 / 2.0
    H[2, 1], H[2, 2] = 1.0 / 6.0, 1.0 / 2.0
    H[3, 1], H[3, 2], H[3, 3] = -1.0 / 2.0, 1.0 / 2.0, 1.0 / 2.0
    H[4, 1], H[4, 2], H[4, 3], H[4, 4] = 3.0 / 2.0, -3.0 / 2.0, 1.0 / 2.0, 1.0 / 2.0
    return A, H


# --------------------------------------------------------------------------------------
# Multistep IMEX (eq. imex and eq. IMEX_adjoint)
# --------------------------------------------------------------------------------------

def multistep_forward(prob, X0, nsteps, dt, order=2):
    """Forward trajectory [X_0, X_1, ..., X_N] of eq. imex."""
    X = [X0]
    Fs = [prob.F(X0)]
    for n in range(1, nsteps + 1):
        a, b, c = sbdf_coeffs(n, order, dt)
        s = len(a) - 1
        R = 0
        for i in range(1, s + 1):
            Xi = X[n - i]
            R = R + c[i] * Fs[n - i] - (a[i] * prob.M(Xi) + b[i] * prob.L(Xi))
        Xn = prob.project(prob.solve(a[0], b[0], R))
        X.append(Xn)
        Fs.append(prob.F(Xn))
    return X


def multistep_tangent(prob, X, dX0, dt, order=2):
    """Tangent (JVP) trajectory [dX_0, ..., dX_N] along the primal trajectory X."""
    nsteps = len(X) - 1
    dX = [dX0]
    for n in range(1, nsteps + 1):
        a, b, c = sbdf_coeffs(n, order, dt)
        s = len(a) - 1
        R = 0
        for i in range(1, s + 1):
            Xi, dXi = X[n - i], dX[n - i]
            R = R + c[i] * prob.F_jvp(Xi, dXi) - (a[i] * prob.M(dXi) + b[i] * prob.L(dXi))
        dX.append(prob.project(prob.solve(a[0], b[0], R)))
    return dX


def multistep_adjoint(prob, X, dJ, dt, order=2):
    """Gradient dJ/dX_0 by eq. IMEX_adjoint run backward over the trajectory X.

    ``dJ(n)`` returns the explicit partial dJ/dX_n (or None).  The adjoint solve
    at step n carries the source dJ/dX_n on its right-hand side wherever the
    objective touches X_n, and the initial condition's cotangent is the
    right-hand side of eq. IMEX_adjoint at n = 0 with no solve (X_0 is an input).
    Superscripts follow the equation: the coefficients of step n+i multiply Y_{n+i}.
    """
    nsteps = len(X) - 1
    Y = [None] * (nsteps + 1)
    coeffs = [None] + [sbdf_coeffs(n, order, dt) for n in range(1, nsteps + 1)]
    for n in range(nsteps, -1, -1):
        lam = dJ(n)
        lam = 0 if lam is None else lam
        for i in range(1, order + 1):
            m = n + i
            if m > nsteps:
                continue
            a, b, c = coeffs[m]
            if i > len(a) - 1:
                continue
            Ym = Y[m]
            lam = lam + c[i] * prob.F_vjp(X[n], Ym) - (a[i] * prob.Mt(Ym) + b[i] * prob.Lt(Ym))
        if n == 0:
            return lam
        a, b, _ = coeffs[n]
        Y[n] = prob.solve_t(a[0], b[0], prob.project(lam))


# --------------------------------------------------------------------------------------
# Runge-Kutta IMEX (Supplementary A.4, RK stage equation and its adjoint)
# --------------------------------------------------------------------------------------

def _dt_of(dt, n):
    """Step size of step n: dt is a scalar (constant step) or a sequence (one per step; the
    stage operators M + dt H_ii L change with it and are factorised per distinct value)."""
    return float(dt[n]) if np.ndim(dt) else float(dt)


def rk_step(prob, Xn, dt, A, H):
    """One RK IMEX step; returns the list of stage values [X_{n,0}, ..., X_{n,s}]."""
    s = A.shape[0] - 1
    stages = [Xn]
    Fst = [prob.F(Xn)]
    MX0 = prob.M(Xn)
    for i in range(1, s + 1):
        R = MX0
        for j in range(i):
            R = R + dt * (A[i, j] * Fst[j] - H[i, j] * prob.L(stages[j]))
        Xi = prob.project(prob.solve(1.0, dt * H[i, i], R))
        stages.append(Xi)
        if i < s:
            Fst.append(prob.F(Xi))
    return stages


def rk_forward(prob, X0, nsteps, dt, A, H):
    """Forward trajectory; returns (states [X_0..X_N], stages per step)."""
    X = [X0]
    stages = []
    for n in range(nsteps):
        st = rk_step(prob, X[-1], _dt_of(dt, n), A, H)
        stages.append(st)
        X.append(st[-1])
    return X, stages


def rk_tangent(prob, stages, dX0, dt, A, H):
    """Tangent trajectory [dX_0, ..., dX_N] along recorded RK stages."""
    s = A.shape[0] - 1
    dX = [dX0]
    for n, st in enumerate(stages):
        dt_n = _dt_of(dt, n)
        dst = [dX[-1]]
        MdX0 = prob.M(dX[-1])
        for i in range(1, s + 1):
            R = MdX0
            for j in range(i):
                R = R + dt_n * (A[i, j] * prob.F_jvp(st[j], dst[j]) - H[i, j] * prob.L(dst[j]))
            dst.append(prob.project(prob.solve(1.0, dt_n * H[i, i], R)))
        dX.append(dst[-1])
    return dX


def rk_adjoint(prob, stages, dJ, dt, A, H):
    """Gradient dJ/dX_0 by the RK IMEX adjoint run backward over recorded stages.

    ``Ybar`` is the total cotangent of the step's output X_{n+1} (the paper's
    Y_{n+1,0}); Y[i] are the stage cotangents solving
    (M + dt H_ii L)^dagger Y_{n,i} = Ybar (i = s) or
    sum_{j>i} dt (A_ji dF/dX_{n,i} - H_ji L)^dagger Y_{n,j} (0 < i < s), and the
    cotangent of X_n is sum_j (M^dagger + dt [A_j0 dF/dX_{n,0} - H_j0 L]^dagger) Y_{n,j}.
    """
    s = A.shape[0] - 1
    nsteps = len(stages)
    Ybar = dJ(nsteps)
    Ybar = 0 * stages[-1][-1] if Ybar is None else Ybar
    for n in range(nsteps - 1, -1, -1):
        st = stages[n]
        dt_n = _dt_of(dt, n)
        Y = [None] * (s + 1)
        Y[s] = prob.solve_t(1.0, dt_n * H[s, s], prob.project(Ybar))
        for i in range(s - 1, 0, -1):
            rhs = 0
            for j in range(i + 1, s + 1):
                rhs = rhs + dt_n * (A[j, i] * prob.F_vjp(st[i], Y[j]) - H[j, i] * prob.Lt(Y[j]))
            Y[i] = prob.solve_t(1.0, dt_n * H[i, i], prob.project(rhs))
        lam = 0
        for j in range(1, s + 1):
            lam = lam + prob.Mt(Y[j]) + dt_n * (A[j, 0] * prob.F_vjp(st[0], Y[j]) - H[j, 0] * prob.Lt(Y[j]))
        src = dJ(n)
        Ybar = lam if src is None else lam + src
    return Ybar


def multistep_adjoint_params(prob, X, dJ, dt, order=2):
    """(dJ/dX_0, dJ/dp) for parameters p of the explicit term.

    F(X_m; p) enters eq. imex of step m + i with weight c_i^{m+i}, so the parameter cotangent
    is sum_m (dF(X_m)/dp)^dagger W_m with W_m = sum_i c_i^{m+i} Y_{m+i}, the same combination
    whose state VJP enters eq. IMEX_adjoint at X_m (eqs. 5-6 with F appearing on the
    right-hand side of the timestepper)."""
    nsteps = len(X) - 1
    Y = [None] * (nsteps + 1)
    coeffs = [None] + [sbdf_coeffs(n, order, dt) for n in range(1, nsteps + 1)]
    gp = 0
    for n in range(nsteps, -1, -1):
        lam = dJ(n)
        lam = 0 if lam is None else lam
        W = 0
        for i in range(1, order + 1):
            m = n + i
            if m > nsteps:
                continue
            a, b, c = coeffs[m]
            if i > len(a) - 1:
                continue
            W = W + c[i] * Y[m]
            lam = lam - (a[i] * prob.Mt(Y[m]) + b[i] * prob.Lt(Y[m]))
        if not isinstance(W, int):
            lam = lam + prob.F_vjp(X[n], W)
            gp = gp + prob.F_param_vjp(X[n], W)
        if n == 0:
            return lam, gp
        a, b, _ = coeffs[n]
        Y[n] = prob.solve_t(a[0], b[0], prob.project(lam))


# --------------------------------------------------------------------------------------
# Time-integrated objectives (Supplementary A.4: a cost depending on a quantity integrated
# over t is handled by adding the ODE dI/dt = J_I to the equation set)
# --------------------------------------------------------------------------------------

class Aug:
    """State of the augmented system: the original coefficient array X and the scalar I."""

    def __init__(self, X, I):
        self.X, self.I = X, complex(I)

    def __add__(self, o):
        if isinstance(o, int) and o == 0:
            return self
        return Aug(self.X + o.X, self.I + o.I)

    __radd__ = __add__

    def __sub__(self, o):
        if isinstance(o, int) and o == 0:
            return self
        return Aug(self.X - o.X, self.I - o.I)

    def __rsub__(self, o):  # 0 - self
        return Aug(-self.X, -self.I)

    def __mul__(self, s):
        return Aug(s * self.X, s * self.I)

    __rmul__ = __mul__


class IntegralObjective:
    """The problem `prob` augmented with dI/dt = g(X): M_aug = diag(M, 1), L_aug = diag(L, 0),
    F_aug(X, I) = (F(X), g(X)), so that the scheme integrates I with the explicit term g and
    J = I_N.  `g_grad(X)` is the gradient of the real functional g under the real inner
    product."""

    def __init__(self, prob, g, g_grad):
        self.p, self.g, self.g_grad = prob, g, g_grad

    def M(self, v):
        return Aug(self.p.M(v.X), v.I)

    def L(self, v):
        return Aug(self.p.L(v.X), 0.0)

    def Mt(self, v):
        return Aug(self.p.Mt(v.X), v.I)

    def Lt(self, v):
        return Aug(self.p.Lt(v.X), 0.0)

    def F(self, v):
        return Aug(self.p.F(v.X), self.g(v.X))

    def F_jvp(self, v, dv):
        return Aug(self.p.F_jvp(v.X, dv.X), inner(self.g_grad(v.X), dv.X))

    def F_vjp(self, v, y):
        return Aug(self.p.F_vjp(v.X, y.X) + y.I.real * self.g_grad(v.X), 0.0)

    def solve(self, a, b, R):
        return Aug(self.p.solve(a, b, R.X), R.I / a)

    def solve_t(self, a, b, R):
        return Aug(self.p.solve_t(a, b, R.X), R.I / a)

    def project(self, v):
        return Aug(self.p.project(v.X), v.I.real)


def integral_gradient(prob, X0, nsteps, dt, g, g_grad, order=2):
    """J = I_N for dI/dt = g(X), I_0 = 0, integrated by the multistep scheme together with the
    state, and dJ/dX_0 by the adjoint of the augmented system (seed dJ/dI_N = 1)."""
    aug = IntegralObjective(prob, g, g_grad)
    V = multistep_forward(aug, Aug(X0, 0.0), nsteps, dt, order)
    J = V[-1].I.real
    seed = Aug(0.0 * X0, 1.0)
    lam = multistep_adjoint(aug, V, lambda n: seed if n == nsteps else None, dt, order)
    return J, lam.X, V


# --------------------------------------------------------------------------------------
# Hessian-vector products (tangent over adjoint, for explicit terms quadratic in X)
# --------------------------------------------------------------------------------------

def multistep_hvp(prob, X, dX, dJ, d2J, dt, order=2):
    """(d^2 J / dX_0^2) v: the tangent, along the trajectory perturbation dX (the tangent of X
    for dX_0 = v), of the adjoint recurrence of multistep_adjoint.  Differentiating
    eq. IMEX_adjoint gives the same recurrence for dY with the extra source
    sum_i c_i^{n+i} d/de[(dF/dX)(X_n + e dX_n)]^dagger Y_{n+i}, which for F quadratic in X is
    F_vjp(dX_n, Y_{n+i}); d2J(n) is the tangent of dJ/dX_n (its Hessian applied to dX_n)."""
    nsteps = len(X) - 1
    Y = [None] * (nsteps + 1)
    dY = [None] * (nsteps + 1)
    coeffs = [None] + [sbdf_coeffs(n, order, dt) for n in range(1, nsteps + 1)]
    for n in range(nsteps, -1, -1):
        lam = dJ(n)
        lam = 0 if lam is None else lam
        dlam = d2J(n)
        dlam = 0 if dlam is None else dlam
        for i in range(1, order + 1):
            m = n + i
            if m > nsteps:
                continue
            a, b, c = coeffs[m]
            if i > len(a) - 1:
                continue
            lam = lam + c[i] * prob.F_vjp(X[n], Y[m]) - (a[i] * prob.Mt(Y[m]) + b[i] * prob.Lt(Y[m]))
            dlam = dlam + c[i] * (prob.F_vjp(X[n], dY[m]) + prob.F_vjp(dX[n], Y[m])) \
                - (a[i] * prob.Mt(dY[m]) + b[i] * prob.Lt(dY[m]))
        if n == 0:
            return dlam
        a, b, _ = coeffs[n]
        Y[n] = prob.solve_t(a[0], b[0], prob.project(lam))
        dY[n] = prob.solve_t(a[0], b[0], prob.project(dlam))
