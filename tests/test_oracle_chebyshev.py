"""Pins for the ultraspherical operators and Gauss-grid Chebyshev transforms
(Sparse spectral methods section; Methods, "Spectral transforms").

Independent references: numpy.polynomial.chebyshev (derivatives, integrals,
evaluation), scipy.special Gegenbauer/Chebyshev-U evaluation, Gauss-Legendre
quadrature for the Gram matrix, and the identity T_n(cos t) = cos(n t).
"""
import numpy as np
import numpy.polynomial.chebyshev as C
import pytest
from scipy.special import eval_chebyu, eval_gegenbauer

from oracle import chebyshev as cb

XS = np.linspace(-0.97, 0.99, 13)


def series_U(c, x):
    return sum(cn * eval_chebyu(n, x) for n, cn in enumerate(c))


def series_C2(c, x):
    return sum(cn * eval_gegenbauer(n, 2.0, x) for n, cn in enumerate(c))


@pytest.mark.parametrize("N", [4, 9, 16])
def test_operators_against_polynomial_library(N):
    rng = np.random.default_rng(N)
    c = rng.standard_normal(N)
    d = rng.standard_normal(N)
    # D0: T -> C1 derivative; S0: T -> C1 conversion
    np.testing.assert_allclose(series_U(cb.D0(N) @ c, XS), C.chebval(XS, C.chebder(c)), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(series_U(cb.S0(N) @ c, XS), C.chebval(XS, c), rtol=1e-12, atol=1e-12)
    # S1: C1 -> C2 conversion
    np.testing.assert_allclose(series_C2(cb.S1(N) @ d, XS), series_U(d, XS), rtol=1e-12, atol=1e-12)
    # D1: derivative of a C1 series, compared through the T basis: U_n = sum of T's
    h = 1e-6
    fd = (series_U(d, XS + h) - series_U(d, XS - h)) / (2 * h)
    np.testing.assert_allclose(series_C2(cb.D1(N) @ d, XS), fd, rtol=1e-6, atol=1e-6)
    # scaled derivative and the T-basis derivative
    np.testing.assert_allclose(cb.deriv_T(N, 2.0) @ c, np.r_[2.0 * C.chebder(c), 0.0], atol=1e-11)


def test_d1_s0_commutation():
    # d/dx (S0 c) in C2 equals S1 (d/dx c) in C2 for T-series c: D1 S0 = S1 D0
    N = 12
    np.testing.assert_allclose(cb.D1(N) @ cb.S0(N), cb.S1(N) @ cb.D0(N), atol=1e-14)


@pytest.mark.parametrize("N", [6, 16, 64])
def test_gauss_transform(N):
    M = 3 * N // 2
    xi = cb.gauss_points(M)
    th = np.arccos(xi)
    Cm = cb.c2g_matrix(N, M)
    for n in [0, 1, N // 2, N - 1]:
        np.testing.assert_allclose(Cm[:, n], np.cos(n * th), atol=1e-13)
    c = np.random.default_rng(N).standard_normal(N)
    np.testing.assert_allclose(cb.g2c_matrix(N, M) @ (Cm @ c), c, atol=1e-13)
    np.testing.assert_allclose(Cm @ c, C.chebval(xi, c), atol=1e-12)
    # a polynomial of degree < N sampled on the grid is reproduced exactly
    p = np.polynomial.Polynomial(np.random.default_rng(1).standard_normal(N))
    np.testing.assert_allclose(C.chebval(xi, cb.g2c_matrix(N, M) @ p(xi)), p(xi), atol=1e-11)


def test_gram_and_integrals():
    N = 10
    x, w = np.polynomial.legendre.leggauss(40)
    T = np.cos(np.outer(np.arccos(x), np.arange(N)))
    np.testing.assert_allclose(cb.gram(N), (T * w[:, None]).T @ T, atol=1e-13)
    for n in range(N):
        e = np.zeros(N)
        e[n] = 1.0
        ci = C.chebint(e)
        np.testing.assert_allclose(cb.integral_weights(N)[n], C.chebval(1, ci) - C.chebval(-1, ci), atol=1e-14)
    bot, top = cb.boundary_rows(N)
    c = np.random.default_rng(2).standard_normal(N)
    assert abs(bot @ c - C.chebval(-1.0, c)) < 1e-13
    assert abs(top @ c - C.chebval(1.0, c)) < 1e-13
