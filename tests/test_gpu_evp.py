"""GPU parity of the shear-flow eigenvalue solver and its adjoint sensitivities (spadj_eigen)
against the oracle's dense QZ eigenpairs and eq. eigenvalue_sens."""
import numpy as np
import pytest
import torch

from oracle.shear_evp import ShearEVP
from paper_2506_14792_gb300 import stability

pytestmark = pytest.mark.gpu

TOL_LAM = 1e-10
TOL_SENS = 1e-9


def _cases(base):
    if base == "poiseuille":
        return [(1.0, 0.0, 10000.0), (1.02056, 0.0, 5772.22), (0.8, 0.3, 3000.0), (1.2, 1.0, 2000.0)]
    return [(1.0, 1.0, 400.0), (0.5, 2.0, 1000.0), (1.5, 0.0, 800.0)]


def _shift_and_iters(lam_all, lam):
    """Shift at a tenth of the gap to the nearest other eigenvalue; enough iterations for the
    two-sided Rayleigh quotient (error ~ rho^(2n)) to reach rounding."""
    others = lam_all[np.abs(lam_all - lam) > 1e-9 * abs(lam)]
    gap = np.min(np.abs(others - lam))
    sigma = lam + 0.1 * gap * (1.0 + 1.0j) / np.sqrt(2.0)
    rho = np.abs(sigma - lam) / np.min(np.abs(others - sigma))
    return sigma, int(np.ceil(np.log(1e-18) / np.log(rho)))


@pytest.mark.parametrize("base", ["poiseuille", "couette"])
def test_eigen_and_sensitivities_match_oracle(base):
    N = 48
    e = ShearEVP(N, base)
    cases = _cases(base)
    P = len(cases)
    want, shifts, iters = [], [], []
    for a, b, Re in cases:
        lam_all, X, Y = e.eigs(a, b, Re)
        lam, Xo, Yo = lam_all[0], X[:, 0], Y[:, 0]
        sens = e.sensitivity(a, b, Re, lam, Xo, Yo)
        sigma, n = _shift_and_iters(lam_all, lam)
        want.append((lam, sens, Xo[:3 * N]))
        shifts.append(sigma)
        iters.append(n)
    prob = stability.shear_evp_problem(N, base, P)
    rng = np.random.default_rng(11)
    x = torch.tensor(rng.standard_normal((P, 3 * N)) + 1j * rng.standard_normal((P, 3 * N))).cuda()
    psi = torch.tensor(rng.standard_normal((P, 3 * N)) + 1j * rng.standard_normal((P, 3 * N))).cuda()
    out = torch.zeros((P, 10), dtype=torch.float64, device="cuda")
    prob.eigen(cases, shifts, max(iters), x, psi, out)
    o = out.cpu().numpy()
    xh = x.cpu().numpy()
    for i, (lam, sens, xo) in enumerate(want):
        got = o[i, 0] + 1j * o[i, 1]
        assert abs(got - lam) <= TOL_LAM * abs(lam), (i, got, lam)
        assert o[i, 8] <= 1e-11 and o[i, 9] <= 1e-11, o[i, 8:]
        for t in range(3):
            g = o[i, 2 + 2 * t] + 1j * o[i, 3 + 2 * t]
            assert abs(g - sens[t]) <= TOL_SENS * abs(sens[t]) + 1e-13 * abs(lam), (i, t, g, sens[t])
        cosang = abs(np.vdot(xh[i], xo)) / (np.linalg.norm(xh[i]) * np.linalg.norm(xo))
        assert cosang >= 1.0 - 1e-12


def test_neutral_curve_newton_matches_oracle():
    """Batched Newton for the neutral Re at several alpha (all alphas in one call per
    iteration) lands where the oracle's Newton does; at alpha_c it is Orszag's Re_c."""
    N = 48
    e = ShearEVP(N, "poiseuille")
    alphas = [0.95, 1.0, 1.02056]
    lam0 = e.leading(1.0, 0.0, 6000.0)[0]
    prob = stability.shear_evp_problem(N, "poiseuille", len(alphas))
    res = stability.neutral_curve(prob, alphas, 6000.0, lam0)
    assert res["newton_iterations"] < 25
    for i, a in enumerate(alphas):
        Re_o, lam_o, d_o = e.neutral_re(a, 6000.0)
        assert abs(res["Re"][i] - Re_o) <= 1e-9 * Re_o, (a, res["Re"][i], Re_o)
        assert abs(res["lam"][i] - lam_o) <= 1e-9 * abs(lam_o)
        assert abs(res["lam"][i].real) <= 1e-11
    assert abs(res["Re"][2] - 5772.22) <= 0.05


def test_full_batch_sampled():
    """152 pencils at N = 64 (one per SM): every pencil converged (residuals), and a sample
    of them against the oracle."""
    N, P = 64, 152
    alphas = np.linspace(0.6, 1.3, 19)
    betas = np.linspace(0.0, 1.4, 8)
    cases = [(a, b, 8000.0) for b in betas for a in alphas]
    e = ShearEVP(N, "poiseuille")
    sample = [0, 37, 90, 151]
    # shifts from the wall-mode branch: lambda ~ -i alpha c with c ~ 0.25
    shifts = [complex(0.0, -0.25 * a) for a, b, _ in cases]
    lam_o = {}
    for i in sample:
        a, b, Re = cases[i]
        lam_all, X, Y = e.eigs(a, b, Re)
        j = int(np.argmin(np.abs(lam_all - shifts[i])))
        lam_o[i] = (lam_all[j], e.sensitivity(a, b, Re, lam_all[j], X[:, j], Y[:, j]))
    prob = stability.shear_evp_problem(N, "poiseuille", P)
    rng = np.random.default_rng(12)
    x = torch.tensor(rng.standard_normal((P, 3 * N)) + 1j * rng.standard_normal((P, 3 * N))).cuda()
    psi = torch.tensor(rng.standard_normal((P, 3 * N)) + 1j * rng.standard_normal((P, 3 * N))).cuda()
    out = torch.zeros((P, 10), dtype=torch.float64, device="cuda")
    prob.eigen(cases, shifts, 200, x, psi, out)
    o = out.cpu().numpy()
    for i in sample:
        lam, sens = lam_o[i]
        got = o[i, 0] + 1j * o[i, 1]
        if max(o[i, 8], o[i, 9]) <= 1e-11:
            assert abs(got - lam) <= TOL_LAM * abs(lam), (i, got, lam)
            g = o[i, 2] + 1j * o[i, 3]
            assert abs(g - sens[0]) <= TOL_SENS * abs(sens[0]), (i, g, sens[0])
        else:  # not converged within 200 iterations: still the nearest eigenvalue to the shift
            assert abs(got - lam) <= 1e-3 * abs(lam)
    assert np.mean(np.max(o[:, 8:10], axis=1) <= 1e-11) >= 0.5


def test_neutral_curve_continuation():
    """Arclength continuation of the neutral curve from the critical point in both directions
    (tangent from the adjoint gradient, minimum-norm Newton back to gamma = 0): every traced
    point is neutral for the oracle's dense eigenproblem, and both branches rise above Re_c."""
    N = 48
    e = ShearEVP(N, "poiseuille")
    a_c = 1.02056
    Re_c, lam_c, _ = e.neutral_re(a_c, 5800.0)
    prob = stability.shear_evp_problem(N, "poiseuille", 2)
    res = stability.trace_neutral_curves(prob, [a_c, a_c], Re_c, lam_c, [1.0, -1.0], ds=0.06, n_points=4)
    A, R = res["alpha"], res["Re"]
    assert np.all(res["newton_steps"] < 20)
    for k in range(1, A.shape[0]):
        for j in range(2):
            lam_o = e.leading(A[k, j], 0.0, R[k, j])[0]
            assert abs(lam_o.real) <= 1e-10, (k, j, A[k, j], R[k, j], lam_o)
    assert np.all(R[1:] > Re_c)
    assert (A[-1, 0] - a_c) * (A[-1, 1] - a_c) < 0  # the two directions go to opposite sides in alpha


def test_largest_chebyshev_size():
    """N = 128 (3N = 384: twelve 32-column chunks per lane, shared memory above the default
    limit) against the oracle."""
    N = 128
    e = ShearEVP(N, "poiseuille")
    cases = [(1.0, 0.0, 10000.0), (0.9, 0.4, 6000.0)]
    shifts, want, iters = [], [], []
    for a, b, Re in cases:
        lam_all, X, Y = e.eigs(a, b, Re)
        sigma, n = _shift_and_iters(lam_all, lam_all[0])
        shifts.append(sigma)
        iters.append(n)
        want.append((lam_all[0], e.sensitivity(a, b, Re, lam_all[0], X[:, 0], Y[:, 0])))
    prob = stability.shear_evp_problem(N, "poiseuille", len(cases))
    rng = np.random.default_rng(13)
    x = torch.tensor(rng.standard_normal((2, 3 * N)) + 1j * rng.standard_normal((2, 3 * N))).cuda()
    psi = torch.tensor(rng.standard_normal((2, 3 * N)) + 1j * rng.standard_normal((2, 3 * N))).cuda()
    out = torch.zeros((2, 10), dtype=torch.float64, device="cuda")
    prob.eigen(cases, shifts, max(iters), x, psi, out)
    o = out.cpu().numpy()
    for i, (lam, sens) in enumerate(want):
        got = o[i, 0] + 1j * o[i, 1]
        assert abs(got - lam) <= TOL_LAM * abs(lam), (i, got, lam)
        for t in range(3):
            g = o[i, 2 + 2 * t] + 1j * o[i, 3 + 2 * t]
            assert abs(g - sens[t]) <= TOL_SENS * abs(sens[t]) + 1e-13 * abs(lam), (i, t, g, sens[t])
