"""Real Fourier collocation transforms and their adjoints (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Methods section, "Spectral transforms": a field has grid values f and
coefficients fhat with fhat = T f and f = T^-1 fhat; the adjoint field
transforms are fhat^dagger = T^-dagger f^dagger and f^dagger = T^dagger
fhat^dagger.  Here ``B`` denotes T^-1 (coefficients -> grid).

Storage (one periodic axis): K complex coefficients c_k, k = 0..K-1, of the
half spectrum of a real field (the Nyquist mode is not stored), sampled on
M >= 2K equispaced points x_j = j L / M (M = 3K for 3/2 dealiasing):

    B c   : g_j = Re c_0 + 2 Re sum_{k=1}^{K-1} c_k exp(2 pi i k j / M)
    T g   : c_k = (1/M) sum_j g_j exp(-2 pi i k j / M),  k < K      (truncation)

With the real inner product over stored reals, <a, b> = Re sum conj(a) b, the
adjoints follow from the definitions (derived in the design notes):

    B^dagger g : (B^dagger g)_0 = sum_j g_j,  (B^dagger g)_k = 2 sum_j g_j exp(-2 pi i k j / M)
    T^dagger c : (T^dagger c)_j = (1/M) Re sum_{k=0}^{K-1} c_k exp(2 pi i k j / M)

numpy's FFT is used as a library primitive for the sums.
"""
import numpy as np


def _pad(c, M):
    """Half spectrum of length M//2+1 holding c_k for k < K and zeros elsewhere."""
    K = c.shape[-1]
    out = np.zeros(c.shape[:-1] + (M // 2 + 1,), dtype=np.complex128)
    out[..., :K] = c
    out[..., 0] = out[..., 0].real
    return out


def c2g(c, M, axis=-1):
    """B: half-spectrum coefficients along ``axis`` -> real grid of M points."""
    c = np.moveaxis(np.asarray(c, dtype=np.complex128), axis, -1)
    g = np.fft.irfft(_pad(c, M), n=M, axis=-1) * M
    return np.moveaxis(g, -1, axis)


def g2c(g, K, axis=-1):
    """T: real grid along ``axis`` -> first K coefficients (3/2-rule truncation)."""
    g = np.moveaxis(np.asarray(g, dtype=np.float64), axis, -1)
    M = g.shape[-1]
    c = np.fft.rfft(g, axis=-1)[..., :K] / M
    return np.moveaxis(c, -1, axis)


def c2g_adj(g, K, axis=-1):
    """B^dagger: grid cotangent -> coefficient cotangent (factor 2 on k >= 1)."""
    g = np.moveaxis(np.asarray(g, dtype=np.float64), axis, -1)
    c = np.fft.rfft(g, axis=-1)[..., :K].copy()
    c[..., 1:] *= 2.0
    c[..., 0] = c[..., 0].real
    return np.moveaxis(c, -1, axis)


def g2c_adj(c, M, axis=-1):
    """T^dagger: coefficient cotangent -> grid cotangent (weight 1/2 on k >= 1)."""
    c = np.moveaxis(np.asarray(c, dtype=np.complex128), axis, -1).copy()
    c[..., 1:] *= 0.5
    g = np.fft.irfft(_pad(c, M), n=M, axis=-1)
    return np.moveaxis(g, -1, axis)


def dense_c2g(K, M):
    """Brute-force real matrix of B acting on [Re c_0, Im c_0, Re c_1, Im c_1, ...]."""
    j = np.arange(M)[:, None]
    k = np.arange(K)[None, :]
    th = 2.0 * np.pi * j * k / M
    w = np.where(k == 0, 1.0, 2.0)
    out = np.zeros((M, 2 * K))
    out[:, 0::2] = w * np.cos(th)
    out[:, 1::2] = -w * np.sin(th)
    out[:, 1] = 0.0  # Im c_0 does not reach the grid
    return out


def dense_g2c(K, M):
    """Brute-force real matrix of T producing [Re c_0, Im c_0, Re c_1, ...]."""
    j = np.arange(M)[None, :]
    k = np.arange(K)[:, None]
    th = 2.0 * np.pi * j * k / M
    out = np.zeros((2 * K, M))
    out[0::2, :] = np.cos(th) / M
    out[1::2, :] = -np.sin(th) / M
    return out


# ---- the same four maps as direct sums over explicit exponentials ----------------------
# Exact in exact arithmetic and equal to the FFT forms above, but with a different order of
# summation (a dense complex matrix product instead of numpy's FFT factorisation).  Used to
# measure how far rounding-order differences alone move a long trajectory and its gradient.

def _expmat(K, M):
    """E[j, k] = exp(2 pi i k j / M), j < M, k < K."""
    j = np.arange(M)[:, None]
    k = np.arange(K)[None, :]
    return np.exp(2j * np.pi * ((j * k) % M) / M)


def c2g_direct(c, M, axis=-1):
    c = np.moveaxis(np.asarray(c, dtype=np.complex128), axis, -1)
    K = c.shape[-1]
    w = np.full(K, 2.0)
    w[0] = 1.0
    g = np.real((c * w) @ _expmat(K, M).T)
    return np.moveaxis(g, -1, axis)


def g2c_direct(g, K, axis=-1):
    g = np.moveaxis(np.asarray(g, dtype=np.float64), axis, -1)
    M = g.shape[-1]
    c = (g @ np.conj(_expmat(K, M))) / M
    return np.moveaxis(c, -1, axis)


def c2g_adj_direct(g, K, axis=-1):
    g = np.moveaxis(np.asarray(g, dtype=np.float64), axis, -1)
    M = g.shape[-1]
    c = g @ np.conj(_expmat(K, M))
    c[..., 1:] *= 2.0
    c[..., 0] = c[..., 0].real
    return np.moveaxis(c, -1, axis)


def g2c_adj_direct(c, M, axis=-1):
    c = np.moveaxis(np.asarray(c, dtype=np.complex128), axis, -1).copy()
    K = c.shape[-1]
    c[..., 0] = c[..., 0].real
    g = np.real(c @ _expmat(K, M).T) / M
    return np.moveaxis(g, -1, axis)


def to_real(c):
    """View a complex coefficient array as the interleaved real state vector."""
    return np.ascontiguousarray(c).view(np.float64)


def from_real(x):
    return np.ascontiguousarray(x, dtype=np.float64).view(np.complex128)
