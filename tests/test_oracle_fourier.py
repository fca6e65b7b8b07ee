"""Pins for the oracle's Fourier collocation transforms (Methods, "Spectral transforms").

The oracle computes B = T^-1 and T with numpy's FFT; these tests fix them with
brute-force cos/sin sums, exact transforms of trigonometric polynomials and the
adjoint identities <B c, g> = <c, B^dagger g>, <T g, c> = <g, T^dagger c>.
"""
import numpy as np
import pytest

from oracle import fourier
from oracle.imex import inner


def _adm(c):
    c = c.copy()
    c[..., 0] = c[..., 0].real
    return c


@pytest.mark.parametrize("K", [2, 4, 6, 8])
def test_dense_bruteforce(K):
    M = 3 * K
    rng = np.random.default_rng(K)
    c = _adm(rng.standard_normal(K) + 1j * rng.standard_normal(K))
    g = rng.standard_normal(M)
    x = fourier.to_real(c)
    np.testing.assert_allclose(fourier.c2g(c, M), fourier.dense_c2g(K, M) @ x, atol=1e-13)
    np.testing.assert_allclose(fourier.to_real(fourier.g2c(g, K)), fourier.dense_g2c(K, M) @ g, atol=1e-14)
    # adjoints are the transposed brute-force matrices
    np.testing.assert_allclose(fourier.to_real(fourier.c2g_adj(g, K)), fourier.dense_c2g(K, M).T @ g, atol=1e-13)
    np.testing.assert_allclose(fourier.g2c_adj(c, M), fourier.dense_g2c(K, M).T @ x, atol=1e-14)


def test_trig_polynomials_exact():
    K, M = 8, 24
    x = 2 * np.pi * np.arange(M) / M
    g = 3.0 + np.cos(3 * x) - 2.0 * np.sin(5 * x)
    c = fourier.g2c(g, K)
    want = np.zeros(K, complex)
    want[0] = 3.0
    want[3] = 0.5
    want[5] = -2.0 / (2j)
    np.testing.assert_allclose(c, want, atol=1e-15)
    np.testing.assert_allclose(fourier.c2g(want, M), g, atol=1e-14)


@pytest.mark.parametrize("K", [4, 64, 128])
def test_roundtrip_and_dot(K):
    M = 3 * K
    rng = np.random.default_rng(10 + K)
    c = _adm(rng.standard_normal((3, K)) + 1j * rng.standard_normal((3, K)))
    g = rng.standard_normal((3, M))
    np.testing.assert_allclose(fourier.g2c(fourier.c2g(c, M), K), c, atol=1e-15 * K)
    for axis_c, axis_g in [(-1, -1)]:
        lhs = inner(fourier.c2g(c, M), g)
        rhs = inner(c, fourier.c2g_adj(g, K))
        assert abs(lhs - rhs) <= 1e-14 * abs(lhs) + 1e-12
        lhs = inner(fourier.g2c(g, K), c)
        rhs = inner(g, fourier.g2c_adj(c, M))
        assert abs(lhs - rhs) <= 1e-14 * abs(lhs) + 1e-14


def test_axis_argument():
    rng = np.random.default_rng(3)
    K, M = 6, 18
    c = _adm(rng.standard_normal((K, 5)).T + 0j).T  # shape (K, 5), transform along axis 0
    c = c + 1j * rng.standard_normal((K, 5))
    c[0] = c[0].real
    g0 = fourier.c2g(c, M, axis=0)
    np.testing.assert_allclose(g0, fourier.c2g(c.T, M).T, atol=1e-14)


def test_direct_sum_transforms_equal_fft_forms_and_brute_force():
    """The direct-sum forms (used to measure rounding-order spread) are the same four maps: they
    agree with the FFT forms and with the brute-force real matrices to rounding."""
    from oracle import fourier as fo
    rng = np.random.default_rng(11)
    for K, M in ((4, 12), (16, 48), (128, 384)):
        c = rng.standard_normal((3, K)) + 1j * rng.standard_normal((3, K))
        g = rng.standard_normal((3, M))
        for a, b, x, n in ((fo.c2g, fo.c2g_direct, c, M), (fo.g2c, fo.g2c_direct, g, K),
                           (fo.c2g_adj, fo.c2g_adj_direct, g, K), (fo.g2c_adj, fo.g2c_adj_direct, c, M)):
            r1, r2 = a(x, n), b(x, n)
            assert np.max(np.abs(r1 - r2)) <= 1e-13 * np.max(np.abs(r1))
        B = fo.dense_c2g(K, M)
        cr = fo.to_real(c[0])
        assert np.allclose(fo.c2g_direct(c[0], M), B @ cr, rtol=0, atol=1e-12 * np.max(np.abs(B @ cr)))
        T = fo.dense_g2c(K, M)
        assert np.allclose(fo.to_real(fo.g2c_direct(g[0], K)), T @ g[0], rtol=0, atol=1e-13)
