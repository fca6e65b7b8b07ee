"""Chebyshev trial basis, ultraspherical test bases and Gauss-grid transforms (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sparse spectral methods section: solutions are expanded in a trial basis (Chebyshev
T_n) and equations are projected onto test bases (ultraspherical C^(1), C^(2)) chosen
so that linear operators become narrowly banded (Olver & Townsend's ultraspherical
method, cited there).  On xi in [-1, 1]:

    d/dxi T_n = n C1_{n-1}                      (D0)
    d/dxi C1_n = 2 C2_{n-1}                     (D1)
    T_0 = C1_0, T_1 = C1_1 / 2, T_n = (C1_n - C1_{n-2}) / 2      (S0)
    C1_n = (C2_n - C2_{n-2}) / (n + 1)                          (S1)

An interval [a, b] is mapped by z = a + (b - a)(xi + 1)/2, which scales each
derivative by 2/(b - a).  All matrices are N x N (coefficients 0..N-1 in, 0..N-1 out).

Transforms use M Gauss-Chebyshev points xi_j = -cos(pi (j + 1/2) / M) (increasing),
with M = 3N/2 for dealiasing (Supplementary B); the matrix transform (Methods:
"transforms implemented directly as matrix multiplications") is

    f(xi_j) = sum_n c_n T_n(xi_j)                 (c2g, M x N matrix)
    c_n = (w_n / M) sum_j f(xi_j) T_n(xi_j),  w_0 = 1, w_n = 2   (g2c, N x M matrix)

by the discrete orthogonality of T_n on Gauss points.
"""
import numpy as np


def D0(N, scale=1.0):
    m = np.zeros((N, N))
    for n in range(1, N):
        m[n - 1, n] = n * scale
    return m


def D1(N, scale=1.0):
    m = np.zeros((N, N))
    for n in range(1, N):
        m[n - 1, n] = 2.0 * scale
    return m


def S0(N):
    m = np.zeros((N, N))
    m[0, 0] = 1.0
    if N > 1:
        m[1, 1] = 0.5
    for n in range(2, N):
        m[n, n] = 0.5
        m[n - 2, n] = -0.5
    return m


def S1(N):
    m = np.zeros((N, N))
    for n in range(N):
        m[n, n] = 1.0 / (n + 1)
        if n >= 2:
            m[n - 2, n] = -1.0 / (n + 1)
    return m


def gauss_points(M):
    return -np.cos(np.pi * (np.arange(M) + 0.5) / M)


def c2g_matrix(N, M):
    """T_n(xi_j), shape (M, N)."""
    xi = gauss_points(M)
    return np.cos(np.outer(np.arccos(xi), np.arange(N)))


def g2c_matrix(N, M):
    """(w_n / M) T_n(xi_j), shape (N, M)."""
    w = np.full(N, 2.0)
    w[0] = 1.0
    return (w[:, None] / M) * c2g_matrix(N, M).T


def deriv_T(N, scale=1.0):
    """Derivative in the T basis: S0^-1 D0 (exact, upper triangular)."""
    return np.linalg.solve(S0(N), D0(N, scale))


def boundary_rows(N):
    """Rows evaluating sum_n c_n T_n at xi = -1 and xi = +1."""
    n = np.arange(N)
    return (-1.0) ** n, np.ones(N)


def integral_weights(N):
    """int_{-1}^{1} T_n dxi = 2 / (1 - n^2) for even n, 0 for odd n."""
    n = np.arange(N)
    w = np.zeros(N)
    even = n % 2 == 0
    w[even] = 2.0 / (1.0 - n[even] ** 2)
    return w


def gram(N):
    """G_mn = int_{-1}^{1} T_m T_n dxi = (I_{m+n} + I_{|m-n|}) / 2 with I_k = int T_k."""
    I = integral_weights(2 * N)
    m = np.arange(N)
    return 0.5 * (I[m[:, None] + m[None, :]] + I[np.abs(m[:, None] - m[None, :])])
