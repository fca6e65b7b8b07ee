"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds input recipes only (random draws, spectral envelopes and
normalisations of the draws); none of the method's arithmetic (transforms,
nonlinear terms, solves, timestepping) lives here.  Every generator is
deterministic in its seed (numpy PCG64).
"""
import numpy as np


def burgers_ic(N, batch=1, seed=1, nmodes=16, length=2.0 * np.pi):
    """Half-spectrum coefficients (batch, N//2) complex of
    u0(x) = sum_{k=1..16} k^-2 (a_k cos kx + b_k sin kx), a_k, b_k ~ N(0,1),
    scaled so that max_x |u0| = 1 (maximum taken on a 1024-point sample grid).
    For N/2 <= 16 only the modes k < N/2 are kept.
    """
    K = N // 2
    rng = np.random.default_rng(seed)
    ab = rng.standard_normal((batch, nmodes, 2))
    nmodes = min(nmodes, K - 1)  # small test sizes keep the modes they can hold
    ab = ab[:, :nmodes]
    k = np.arange(1, nmodes + 1)
    c = np.zeros((batch, K), dtype=np.complex128)
    c[:, 1:nmodes + 1] = (ab[:, :, 0] - 1j * ab[:, :, 1]) * (0.5 / k ** 2)
    xs = np.arange(1024) * (2.0 * np.pi / 1024)
    cosm = np.cos(np.outer(k, xs))
    sinm = np.sin(np.outer(k, xs))
    for s in range(0, batch, 2048):
        a = ab[s:s + 2048, :, 0] / k ** 2
        b = ab[s:s + 2048, :, 1] / k ** 2
        u = a @ cosm + b @ sinm
        c[s:s + 2048] /= np.max(np.abs(u), axis=1)[:, None]
    return c


def random_coeffs(shape, seed, scale=1.0):
    """Complex N(0, scale^2) coefficients (used for test directions and cotangents)."""
    rng = np.random.default_rng(seed)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def rb_ic(Nx, Nz, seed=2, amp=1e-3):
    """Rayleigh-Benard initial state (3, Nx/2, Nz) complex: u = w = 0 and a temperature
    perturbation theta = amp * sum a_{m,n} phi_n(z) e^{i kx_m x} with N(0,1) draws a_{m,n},
    phi_n = T_{n+2} - T_n (vanishing at both walls), a (1 + n)^-2 (1 + m)^-1 envelope and
    Hermitian-consistent mean pencil (real coefficients at m = 0)."""
    K = Nx // 2
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((K, Nz - 2)) + 1j * rng.standard_normal((K, Nz - 2))
    a[0] = a[0].real
    env = 1.0 / ((1.0 + np.arange(Nz - 2))[None, :] ** 2 * (1.0 + np.arange(K))[:, None])
    a *= env
    th = np.zeros((K, Nz), dtype=np.complex128)
    th[:, 2:] += a
    th[:, :Nz - 2] -= a
    s = np.zeros((3, K, Nz), dtype=np.complex128)
    s[2] = amp * th
    return s


def kolmogorov_ic(N, seed, urms=1.0):
    """Vorticity coefficients [N/2][N] complex (layout of the Kolmogorov problem: kx half
    spectrum, ky in FFT order, ky = -N/2 row zero, kx = 0 column Hermitian) with velocity
    energy spectrum E(k) ~ k^-3 for 1 <= |k| <= N/3 (|w_k| ~ 1/|k|), random phases, scaled
    to rms velocity `urms` (Parseval over the Hermitian-completed spectrum)."""
    Kx = N // 2
    rng = np.random.default_rng(seed)
    kx = np.arange(Kx)[:, None]
    ky = np.fft.fftfreq(N, 1.0 / N)[None, :]
    k = np.sqrt(kx ** 2 + ky ** 2)
    band = (k >= 1.0) & (k <= N / 3.0) & (ky != -N // 2)
    phase = np.exp(2j * np.pi * rng.random((Kx, N)))
    w = np.where(band, phase / np.where(k > 0, k, 1.0), 0.0)
    # Hermitian kx = 0 column: w(0, -ky) = conj w(0, ky)
    col = w[0].copy()
    neg = np.concatenate([[0], np.arange(N - 1, 0, -1)])
    half = (ky[0] > 0)
    col[neg[half]] = np.conj(col[half])
    col[0] = 0.0
    w[0] = col
    # rms velocity^2 = sum over the full spectrum of |w|^2 / |k|^2 (kx >= 1 counted twice)
    weight = np.where(kx == 0, 1.0, 2.0)
    e = np.sum(weight * np.abs(w) ** 2 / np.where(k > 0, k, 1.0) ** 2)
    return w * (urms / np.sqrt(e))


def kolmogorov_batch(sizes, seeds):
    """List of per-member ICs for a mixed-resolution batch."""
    return [kolmogorov_ic(n, s) for n, s in zip(sizes, seeds)]


def cnn_params(seed, scale_out=0.1):
    """Seeded initial weights of the 1-32-32-32-1 closure CNN: N(0, 1/fan_in) weights, zero
    biases, last layer scaled by `scale_out` (flat vector, layer by layer: W then b)."""
    rng = np.random.default_rng(seed)
    ch = (1, 32, 32, 32, 1)
    parts = []
    for k, (ci, co) in enumerate(zip(ch[:-1], ch[1:])):
        W = rng.standard_normal((co, ci, 3, 3)) / np.sqrt(9.0 * ci)
        if k == 3:
            W *= scale_out
        parts += [W.ravel(), np.zeros(co)]
    return np.concatenate(parts)


def couette_ic(Nx, Ny, Nz, seed=5, norm=1e-4, Lx=4.0 * np.pi, Ly=2.0 * np.pi, nz0=6):
    """Plane-Couette initial velocity (3, Nx/2, Ny, Nz) complex (u, v, w; kx half spectrum,
    ky in FFT order, Chebyshev T_n in z on [-1, 1]).

    u0 = curl(Psi (1 - z^2)^2) with a random vector potential Psi whose (kx, ky) coefficients
    are N(0,1) draws times |k_h|^-2 for 0 < |k_h|, kx index <= Nx/4, |ky| <= Ny/4, and whose z
    dependence is a Chebyshev series of degree < nz0 with a 2^-n envelope; the (1 - z^2)^2
    factor makes u0 vanish at both walls and the curl makes it divergence-free.  The ky = -Ny/2
    row is zero and the kx = 0 plane Hermitian.  Scaled to the volume-averaged norm
    ((1/V) int |u0|^2 dV)^(1/2) = `norm`.  Polynomial products, derivatives and integrals in z
    use numpy.polynomial.chebyshev; the degree stays below Nz so the field is exact."""
    from numpy.polynomial import chebyshev as C
    Kx, N = Nx // 2, Nz
    nz0 = max(1, min(nz0, N - 5))
    rng = np.random.default_rng(seed)
    alpha = 2.0 * np.pi / Lx * np.arange(Kx)
    kyi = np.fft.fftfreq(Ny, 1.0 / Ny).astype(int)
    beta = 2.0 * np.pi / Ly * kyi
    draw = rng.standard_normal((3, Kx, Ny, nz0)) + 1j * rng.standard_normal((3, Kx, Ny, nz0))
    kh = np.sqrt(alpha[:, None] ** 2 + beta[None, :] ** 2)
    band = (np.arange(Kx)[:, None] <= Nx // 4) & (np.abs(kyi)[None, :] <= Ny // 4) & (kh > 0)
    band &= (kyi != -(Ny // 2))[None, :]
    env = np.where(band, 1.0 / np.where(kh > 0, kh, 1.0) ** 2, 0.0)
    psi = draw * env[None, :, :, None] * (0.5 ** np.arange(nz0))[None, None, None, :]
    # Hermitian kx = 0 plane: psi(0, -ky) = conj psi(0, ky)
    neg = np.concatenate([[0], np.arange(Ny - 1, 0, -1)])
    pos = kyi > 0
    psi[:, 0, neg[pos]] = np.conj(psi[:, 0, pos])
    psi[:, 0, 0] = psi[:, 0, 0].real
    bump = C.poly2cheb([1.0, 0.0, -2.0, 0.0, 1.0])  # (1 - z^2)^2

    def series(c):  # Chebyshev coefficients (..., deg) -> (..., N) of c * bump
        out = np.zeros(c.shape[:-1] + (N,), dtype=np.complex128)
        for idx in np.ndindex(c.shape[:-1]):
            if np.any(c[idx] != 0):
                p = C.chebmul(c[idx], bump)
                out[idx][:len(p)] = p
        return out

    def dz(c):
        out = np.zeros_like(c)
        for idx in np.ndindex(c.shape[:-1]):
            d = C.chebder(c[idx])
            out[idx][:len(d)] = d
        return out

    P = series(psi)                      # Psi (1 - z^2)^2, (3, Kx, Ny, N)
    ia = 1j * alpha[:, None, None]
    ib = 1j * beta[None, :, None]
    u = np.stack([ib * P[2] - dz(P[1]), dz(P[0]) - ia * P[2], ia * P[1] - ib * P[0]])
    # (1/V) int |u|^2 dV = 1/2 sum_{kx, ky} w_kx int_{-1}^{1} |u_hat(z)|^2 dz, w = 1 (kx = 0), 2
    wk = np.where(np.arange(Kx) == 0, 1.0, 2.0)
    e = 0.0
    for f in range(3):
        for m in range(Kx):
            for j in range(Ny):
                c = u[f, m, j]
                if np.any(c != 0):
                    sq = C.chebadd(C.chebmul(c.real, c.real), C.chebmul(c.imag, c.imag))
                    I = C.chebint(sq)
                    e += 0.5 * wk[m] * (C.chebval(1.0, I) - C.chebval(-1.0, I))
    return u * (norm / np.sqrt(e))
