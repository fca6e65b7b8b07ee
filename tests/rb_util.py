"""Shared helpers for the Rayleigh-Benard GPU parity tests (oracle-side conversions)."""
import numpy as np


def gpu_problem(Nx, Nz, Ra=1e6, Pr=1.0, dt=1e-3, nonlinear=True, Lx=4.0, scheme=None):
    from paper_2506_14792_gb300 import spadj
    sch = spadj.SPADJ_RK222 if scheme is None else scheme
    return spadj.Problem(spadj.SPADJ_RB2D, sch, [Nx, Nz], [Lx], [Ra, Pr], dt, nonlinear=nonlinear)


def F_T(o, X):
    """Oracle nonlinear term in Chebyshev-T space: the C^(2) rows of F are S1S0 F_T."""
    Fe = o.F(X)
    N = o.N
    return np.stack([np.linalg.solve(o.SS, Fe[:, f * N:(f + 1) * N].T).T for f in range(3)])


def F_T_jvp(o, X, dX):
    Fe = o.F_jvp(X, dX)
    N = o.N
    return np.stack([np.linalg.solve(o.SS, Fe[:, f * N:(f + 1) * N].T).T for f in range(3)])


def F_T_vjp(o, X, fbar):
    """(dF_T/dX)^dagger fbar = F_vjp(X, Y) with the C^(2) rows of Y = S1S0^-T fbar."""
    N = o.N
    Y = np.zeros((o.Kx, o.nvar), complex)
    for f in range(3):
        Y[:, f * N:(f + 1) * N] = np.linalg.solve(o.SS.T, fbar[f].T).T
    return o.state(o.F_vjp(X, Y))


def stage_solve(o, v, b, transpose=False):
    """Prognostic part of (M + b L)^-1 [S1S0 v; 0] (or the adjoint map)."""
    N = o.N
    if not transpose:
        R = np.zeros((o.Kx, o.nvar), complex)
        for f in range(3):
            R[:, f * N:(f + 1) * N] = v[f] @ o.SS.T
        return o.state(o.project(o.solve(1.0, b, R)))
    R = o.project(o.pencils(v))
    Y = o.solve_t(1.0, b, R)
    return np.stack([Y[:, f * N:(f + 1) * N] @ o.SS for f in range(3)])
