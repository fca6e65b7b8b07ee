"""Pins for the shear-flow eigenvalue oracle and its adjoint eigenvalue sensitivities.

* Plane Poiseuille flow: the least stable 2D eigenvalue at alpha = 1, Re = 10000 and the
  critical point of the neutral curve (Re_c, alpha_c, phase speed) from Orszag (1971), the
  study the paper's Parametric sensitivity example reproduces (tests/golden).  At the
  critical point the neutral curve has its nose, so dgamma/dalpha = 0 there: a pin of the
  alpha-sensitivity independent of any finite difference.
* Base-flow products: [U T_n] and [U' T_n] against numpy's Chebyshev product and
  derivative followed by the S1 S0 conversion.
* Plane Couette base: the pencil equals the Couette oracle's (pinned there by an independent
  collocation Orr-Sommerfeld/Squire solver), and every pencil is linearly stable (Romanov).
* Sensitivities (eq. eigenvalue_sens) against central finite differences of the eigenvalue;
  dL/dp against exact central differences (L is quadratic in alpha, beta); the adjoint
  eigenvector solves the adjoint problem; dlambda/dbeta = 0 at beta = 0 (reflection y -> -y).
* Shift-invert operator: 1/(sigma - lambda) is an eigenvalue of its prognostic block.
"""
import os

import numpy as np
import numpy.polynomial.chebyshev as C
import pytest

from oracle import chebyshev as cb
from oracle import couette as co
from oracle.shear_evp import ShearEVP

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "orszag1971_poiseuille.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_orszag_least_stable_eigenvalue():
    g = _golden()
    e = ShearEVP(80, "poiseuille")
    lam, X, Y = e.leading(g["alpha"], 0.0, g["Re"])
    c = 1j * lam / g["alpha"]  # lambda = -i alpha c
    assert abs(c.real - g["c_r"]) <= 2e-11
    assert abs(c.imag - g["c_i"]) <= 2e-11


def test_orszag_critical_point_and_nose():
    """Newton in Re (dgamma/dRe from the adjoint) at alpha_c lands on Re_c; the phase speed
    matches, and dgamma/dalpha vanishes at the nose of the neutral curve (while it is O(1e-2)
    a few per cent of alpha away from it)."""
    g = _golden()
    e = ShearEVP(64, "poiseuille")
    Re, lam, d = e.neutral_re(g["alpha_c"], 5800.0)
    assert abs(lam.real) <= 1e-13
    assert abs(Re - g["Re_c"]) <= 0.01
    assert abs(-lam.imag / g["alpha_c"] - g["c_crit"]) <= 1e-5
    assert abs(d[1].real) <= 2e-5
    Re2, lam2, d2 = e.neutral_re(0.95, 6000.0)
    assert Re2 > g["Re_c"] + 100 and d2[1].real > 1e-2


@pytest.mark.parametrize("base", ["couette", "poiseuille"])
def test_base_flow_products(base):
    N = 12
    e = ShearEVP(N, base)
    U = [0.0, 1.0] if base == "couette" else [0.5, 0.0, -0.5]  # z, 1 - z^2 in T
    rng = np.random.default_rng(3)
    c = rng.standard_normal(N)
    ext = N + 2
    conv = (cb.S1(ext) @ cb.S0(ext))
    pad = lambda v: np.concatenate([v, np.zeros(ext - len(v))])
    want_U = (conv @ pad(C.chebmul(U, c)))[:N]
    want_UP = (conv @ pad(C.chebmul(C.chebder(U), c)))[:N]
    np.testing.assert_allclose(e.Umat @ c, want_U, atol=1e-13)
    np.testing.assert_allclose(e.UPmat @ c, want_UP, atol=1e-13)


def test_couette_base_equals_couette_pencil_and_is_stable():
    o = co.Couette(8, 4, 24, 1000.0)
    e = ShearEVP(24, "couette")
    for m, j in ((1, 0), (1, 1), (2, 3), (3, 1)):
        Mo, Lo = o.pencil_matrices(o.alpha[m], o.beta[j])
        Me, Le = e.matrices(o.alpha[m], o.beta[j], 1000.0)
        assert np.array_equal(Mo, Me) and np.array_equal(Lo, Le)
        assert e.leading(o.alpha[m], o.beta[j], 1000.0)[0].real < 0


@pytest.mark.parametrize("base,a,b,Re", [("poiseuille", 1.0, 0.5, 3000.0), ("couette", 1.0, 1.0, 400.0)])
def test_sensitivity_vs_central_differences(base, a, b, Re):
    e = ShearEVP(40, base)
    lam, X, Y = e.leading(a, b, Re)
    s = e.sensitivity(a, b, Re, lam, X, Y)
    p0 = np.array([Re, a, b])
    for i, h in enumerate((1e-4 * Re, 1e-5, 1e-5)):
        pp, pm = p0.copy(), p0.copy()
        pp[i] += h
        pm[i] -= h
        lp = e.leading(pp[1], pp[2], pp[0], target=lam)[0]
        lm = e.leading(pm[1], pm[2], pm[0], target=lam)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - s[i]) <= 1e-6 * abs(s[i]), (i, fd, s[i])


def test_dL_and_adjoint_eigenvector():
    e = ShearEVP(20, "poiseuille")
    a, b, Re = 0.8, 0.3, 2000.0
    dRe, da, db = e.dL(a, b, Re)
    h = 1e-3
    for i, D in ((1, da), (2, db)):  # L is quadratic in alpha and beta: central difference exact
        pp, pm = [Re, a, b], [Re, a, b]
        pp[i] += h
        pm[i] -= h
        fd = (e.matrices(pp[1], pp[2], pp[0])[1] - e.matrices(pm[1], pm[2], pm[0])[1]) / (2 * h)
        assert np.max(np.abs(fd - D)) <= 1e-9 * np.max(np.abs(D))
    hR = 1e-3 * Re
    fd = (e.matrices(a, b, Re + hR)[1] - e.matrices(a, b, Re - hR)[1]) / (2 * hR)
    assert np.max(np.abs(fd - dRe)) <= 1e-5 * np.max(np.abs(dRe))
    Mm, Lm = e.matrices(a, b, Re)
    lam, X, Y = e.leading(a, b, Re)
    scale = np.max(np.abs(Lm)) + abs(lam) * np.max(np.abs(Mm))
    assert np.linalg.norm(lam * Mm @ X + Lm @ X) <= 1e-10 * scale * np.linalg.norm(X)
    assert np.linalg.norm(np.conj(lam) * Mm.conj().T @ Y + Lm.conj().T @ Y) <= 1e-10 * scale * np.linalg.norm(Y)


def test_beta_reflection():
    e = ShearEVP(24, "poiseuille")
    lam_p = e.leading(1.0, 0.4, 3000.0)[0]
    lam_m = e.leading(1.0, -0.4, 3000.0)[0]
    assert abs(lam_p - lam_m) <= 1e-11 * abs(lam_p)
    lam, X, Y = e.leading(1.0, 0.0, 3000.0)
    assert abs(e.sensitivity(1.0, 0.0, 3000.0, lam, X, Y)[2]) <= 1e-12


def test_shift_invert_spectrum():
    e = ShearEVP(24, "poiseuille")
    a, b, Re = 1.0, 0.0, 5000.0
    lam = e.leading(a, b, Re)[0]
    sigma = lam + 0.02 + 0.01j
    mu = np.linalg.eigvals(e.shift_invert(a, b, Re, sigma))
    want = 1.0 / (sigma - lam)
    assert np.min(np.abs(mu - want)) <= 1e-9 * abs(want)
    assert np.argmax(np.abs(mu)) == np.argmin(np.abs(mu - want))


def test_channel_pencils_of_the_3d_problem():
    """The 3D problem's channel option assembles the Poiseuille pencils pinned above."""
    o = co.Couette(8, 4, 20, 2000.0, base="poiseuille")
    e = ShearEVP(20, "poiseuille")
    for m, j in ((1, 0), (1, 1), (3, 2), (0, 1)):
        Mo, Lo = o.pencil_matrices(o.alpha[m], o.beta[j])
        Me, Le = e.matrices(o.alpha[m], o.beta[j], 2000.0)
        np.testing.assert_allclose(Lo, Le, rtol=0, atol=1e-14)
        np.testing.assert_array_equal(Mo, Me)
