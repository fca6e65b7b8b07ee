"""Neutral stability curves of plane shear flows with adjoint eigenvalue sensitivities.

Parametric sensitivity example: at each streamwise wavenumber alpha, Newton's method in Re
drives the growth rate gamma = Re(lambda) of the least stable eigenvalue to zero, with
dgamma/dRe = Re(dlambda/dRe) from the adjoint sensitivity (eq. eigenvalue_sens).  Every alpha
of the curve advances together: one ``spadj_eigen`` call per Newton iteration factorises the
shifted pencils (shift = the previous eigenvalue plus a small offset, so the shift-invert
iteration locks onto the same mode) and runs the forward and adjoint iterations and the
sensitivities on the GPU.  The previous eigenvectors seed the next iteration.  This module
only steers the iteration; all eigen-arithmetic runs in the library.
"""
import numpy as np

from . import spadj


def _shift(lam, rel):
    return lam + rel * np.maximum(np.abs(lam), 1e-3) * (1.0 + 1.0j)


def neutral_curve(prob, alphas, Re0, lam0, beta=0.0, n_iter=30, tol=1e-10, max_newton=25, shift_rel=2e-3,
                  seed=0):
    """Re on the neutral curve gamma_max(Re, alpha) = 0 for every alpha.

    prob: a SPADJ_SHEAR_EVP ``spadj.Problem`` with batch >= len(alphas); Re0, lam0: starting
    Reynolds numbers and eigenvalue guesses (scalars or one per alpha).  Returns a dict with
    Re, lam, dlam (P x 3: d/dRe, d/dalpha, d/dbeta), residuals and the Newton iterations used.
    """
    import torch
    alphas = np.asarray(alphas, dtype=np.float64).reshape(-1)
    P = alphas.size
    Re = np.broadcast_to(np.asarray(Re0, dtype=np.float64), (P,)).copy()
    lam = np.broadcast_to(np.asarray(lam0, dtype=np.complex128), (P,)).copy()
    H = 3 * prob.desc.n[2]
    g = torch.Generator(device="cpu").manual_seed(seed)
    x = torch.randn((P, H), dtype=torch.complex128, generator=g).cuda()
    psi = torch.randn((P, H), dtype=torch.complex128, generator=g).cuda()
    out = torch.zeros((P, 10), dtype=torch.float64, device="cuda")
    done = np.zeros(P, dtype=bool)
    it = 0
    for it in range(1, max_newton + 1):
        prm = np.stack([alphas, np.full(P, float(beta)), Re], axis=1)
        prob.eigen(prm, _shift(lam, shift_rel), n_iter, x, psi, out)
        o = out.cpu().numpy()
        lam = o[:, 0] + 1j * o[:, 1]
        dRe = o[:, 2]
        step = np.where(done, 0.0, lam.real / dRe)
        Re = Re - step
        done |= np.abs(step) <= tol * np.abs(Re)
        if done.all():
            break
    prm = np.stack([alphas, np.full(P, float(beta)), Re], axis=1)
    prob.eigen(prm, _shift(lam, shift_rel), n_iter, x, psi, out)
    o = out.cpu().numpy()
    return {
        "alpha": alphas,
        "Re": Re,
        "lam": o[:, 0] + 1j * o[:, 1],
        "dlam": np.stack([o[:, 2] + 1j * o[:, 3], o[:, 4] + 1j * o[:, 5], o[:, 6] + 1j * o[:, 7]], axis=1),
        "residual": o[:, 8:10].copy(),
        "newton_iterations": it,
    }


def trace_neutral_curves(prob, alpha0, Re0, lam0, directions, ds, n_points, beta=0.0, n_iter=30, tol=1e-12,
                         max_newton=20, shift_rel=2e-3, seed=0):
    """Continuation of neutral curves gamma_max(alpha, Re) = 0 (Parametric sensitivity example):
    from the neutral points (alpha0, Re0) (one per curve, eigenvalues lam0), each curve steps by
    ds along the tangent of the curve in (alpha, log Re), which the adjoint gradient
    (dgamma/dalpha, Re dgamma/dRe) gives, in the given direction (+1 or -1), and returns to the
    curve by Newton steps along the gradient (the minimum-norm correction).  All curves advance
    together, one spadj_eigen call per Newton step.  Returns arrays of shape (n_points + 1, P):
    alpha, Re, lam, and the Newton steps each point took.  Turning points in Re are crossed
    without special treatment, because the parametrisation is by arclength."""
    import torch
    a = np.asarray(alpha0, dtype=np.float64).reshape(-1).copy()
    P = a.size
    r = np.log(np.broadcast_to(np.asarray(Re0, dtype=np.float64), (P,)).copy())
    lam = np.broadcast_to(np.asarray(lam0, dtype=np.complex128), (P,)).copy()
    sgn = np.broadcast_to(np.asarray(directions, dtype=np.float64), (P,)).copy()
    H = 3 * prob.desc.n[2]
    g = torch.Generator(device="cpu").manual_seed(seed)
    x = torch.randn((P, H), dtype=torch.complex128, generator=g).cuda()
    psi = torch.randn((P, H), dtype=torch.complex128, generator=g).cuda()
    out = torch.zeros((P, 10), dtype=torch.float64, device="cuda")

    def evaluate(a_, r_, lam_):
        prm = np.stack([a_, np.full(P, float(beta)), np.exp(r_)], axis=1)
        prob.eigen(prm, _shift(lam_, shift_rel), n_iter, x, psi, out)
        o = out.cpu().numpy()
        lam_n = o[:, 0] + 1j * o[:, 1]
        grad = np.stack([o[:, 4], o[:, 2] * np.exp(r_)], axis=1)  # (dgamma/dalpha, dgamma/dlog Re)
        return lam_n, grad

    def correct(a_, r_, lam_):
        steps = np.zeros(P, dtype=int)
        for _ in range(max_newton):
            lam_, grad = evaluate(a_, r_, lam_)
            gam = lam_.real
            if np.all(np.abs(gam) <= tol):
                break
            n2 = np.sum(grad * grad, axis=1)
            act = np.abs(gam) > tol
            a_ = a_ - np.where(act, gam * grad[:, 0] / n2, 0.0)
            r_ = r_ - np.where(act, gam * grad[:, 1] / n2, 0.0)
            steps += act
        return a_, r_, lam_, grad, steps

    a, r, lam, grad, st = correct(a, r, lam)
    A, R, L, S = [a.copy()], [np.exp(r)], [lam.copy()], [st]
    for _ in range(n_points):
        t = np.stack([-grad[:, 1], grad[:, 0]], axis=1)
        t /= np.linalg.norm(t, axis=1, keepdims=True)
        a_p = a + sgn * ds * t[:, 0]
        r_p = r + sgn * ds * t[:, 1]
        a, r, lam, grad, st = correct(a_p, r_p, lam)
        A.append(a.copy()); R.append(np.exp(r)); L.append(lam.copy()); S.append(st)
    return {"alpha": np.array(A), "Re": np.array(R), "lam": np.array(L), "newton_steps": np.array(S)}


def shear_evp_problem(N, base="poiseuille", max_pencils=1):
    """A SPADJ_SHEAR_EVP problem with N Chebyshev modes for plane Couette or Poiseuille flow."""
    b = {"couette": 0, "poiseuille": 1}[base]
    return spadj.Problem(spadj.SPADJ_SHEAR_EVP, 0, (0, 0, N), (0.0, 0.0, 0.0), (b,), 1.0, batch=max_pencils)
