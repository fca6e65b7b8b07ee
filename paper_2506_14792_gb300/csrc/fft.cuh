// FP64 shared-memory FFTs for the collocation transforms (Methods, "Spectral transforms").
//
// A real field of M = 2L grid points is transformed through one complex FFT of length
// L on the packed sequence z_j = g_{2j} + i g_{2j+1} (the classic half-length real FFT),
// so a 3/2-dealiased grid of 384 points costs one 192-point complex FFT.  The complex
// FFT is a Stockham autosort (ping-pong between two shared buffers, natural order in
// and out) with radix-4/3/2 passes; all threads of the CTA take part and every pass
// ends with a CTA barrier.  Twiddles come from a device table
//   WM[m] = exp(-2 pi i m / M),  m = 0..M-1,
// whose even entries are the L-point twiddles exp(-2 pi i m / L).
#pragma once
#include <cuda_runtime.h>

namespace spadj {

struct FFTPlan {
  int n;        // complex length L
  int nrad;     // number of passes
  int rad[8];   // radix of each pass (product = n)
};

// Factor n = 2^a 3^b into radix-4 passes, then one radix-2 if a is odd, then radix-3.
inline FFTPlan make_plan(int n) {
  FFTPlan p{};
  p.n = n;
  int m = n;
  while (m % 4 == 0) { p.rad[p.nrad++] = 4; m /= 4; }
  if (m % 2 == 0) { p.rad[p.nrad++] = 2; m /= 2; }
  while (m % 3 == 0) { p.rad[p.nrad++] = 3; m /= 3; }
  if (m != 1) p.nrad = -1;  // unsupported length
  return p;
}

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// multiply by i*s (s = +-1)
__device__ __forceinline__ double2 cmul_i(double2 a, double s) { return make_double2(-s * a.y, s * a.x); }

// Packed-spectrum entry of a real inverse transform, e + i d conj(w), written as two multiply-add
// chains (the FP64 pipe is the binding resource: 8 instructions per entry instead of 10).
__device__ __forceinline__ double2 c2r_combine(double2 e, double2 d, double2 w) {
  return make_double2(fma(d.x, w.y, fma(-d.y, w.x, e.x)), fma(d.x, w.x, fma(d.y, w.y, e.y)));
}

// Twice the spectrum entry of a real forward transform from the packed FFT value zk and
// zc = conj(z_{L-k}): (zk + zc) - i (zk - zc) w as multiply-add chains (8 instructions; the
// factor 1/2 is left to the caller's scaling).
__device__ __forceinline__ double2 r2c_combine2(double2 zk, double2 zc, double2 w) {
  const double sx = zk.x + zc.x, sy = zk.y + zc.y, dx = zk.x - zc.x, dy = zk.y - zc.y;
  return make_double2(fma(dy, w.x, fma(dx, w.y, sx)), fma(dy, w.y, fma(-dx, w.x, sy)));
}
// The spectrum entry itself: r2c_combine2 / 2.
__device__ __forceinline__ double2 r2c_combine(double2 zk, double2 zc, double2 w) {
  return cscale(r2c_combine2(zk, zc, w), 0.5);
}

// Twiddle exp(SIGN * 2 pi i m / L) from the M-table (M = 2L): entry 2m, conjugated for SIGN=+1.
template <int SIGN>
__device__ __forceinline__ double2 twL(const double2* __restrict__ WM, int m) {
  double2 w = __ldg(&WM[2 * m]);
  return SIGN > 0 ? cconj(w) : w;
}
// SIGN * i * a (exact: a swap and a sign change, no multiply)
template <int SIGN>
__device__ __forceinline__ double2 rot(double2 a) {
  return SIGN > 0 ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

// Complex FFT of length p.n held in buffer a (b is scratch of the same size).  SIGN = -1:
// forward exp(-), SIGN = +1: inverse exp(+) (unnormalised).  Returns the buffer holding
// the result (a or b).  All threads of the CTA must call it; it synchronises internally
// and on return the result is visible to every thread.
template <int SIGN>
static __device__ __noinline__ double2* cfft_smem_t(double2* a, double2* b, const FFTPlan p,
                                                    const double2* __restrict__ WM) {
  const int n = p.n;
  const int tid = threadIdx.x, nt = blockDim.x;
  int Ns = 1;
  for (int pass = 0; pass < p.nrad; ++pass) {
    const int R = p.rad[pass];
    const int nb = n / R;
    const int tstep = n / (Ns * R);  // twiddle index stride in L-units
    for (int j = tid; j < nb; j += nt) {
      const int k = j % Ns;
      const int base = (j - k) * R + k;
      if (R == 4) {
        double2 v0 = a[j], v1 = a[j + nb], v2 = a[j + 2 * nb], v3 = a[j + 3 * nb];
        if (k) {
          v1 = cmul(v1, twL<SIGN>(WM, k * tstep));
          v2 = cmul(v2, twL<SIGN>(WM, 2 * k * tstep));
          v3 = cmul(v3, twL<SIGN>(WM, 3 * k * tstep));
        }
        const double2 t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3);
        const double2 t3 = rot<SIGN>(csub(v1, v3));
        b[base] = cadd(t0, t2);
        b[base + Ns] = cadd(t1, t3);
        b[base + 2 * Ns] = csub(t0, t2);
        b[base + 3 * Ns] = csub(t1, t3);
      } else if (R == 2) {
        double2 v0 = a[j], v1 = a[j + nb];
        if (k) v1 = cmul(v1, twL<SIGN>(WM, k * tstep));
        b[base] = cadd(v0, v1);
        b[base + Ns] = csub(v0, v1);
      } else {  // R == 3
        double2 v0 = a[j], v1 = a[j + nb], v2 = a[j + 2 * nb];
        if (k) {
          v1 = cmul(v1, twL<SIGN>(WM, k * tstep));
          v2 = cmul(v2, twL<SIGN>(WM, 2 * k * tstep));
        }
        const double h = 0.86602540378443864676;  // sqrt(3)/2
        const double2 t = cadd(v1, v2);
        const double2 m = make_double2(fma(-0.5, t.x, v0.x), fma(-0.5, t.y, v0.y));
        const double2 r = rot<SIGN>(csub(v1, v2));  // m +- h r as multiply-adds
        b[base] = cadd(v0, t);
        b[base + Ns] = make_double2(fma(h, r.x, m.x), fma(h, r.y, m.y));
        b[base + 2 * Ns] = make_double2(fma(-h, r.x, m.x), fma(-h, r.y, m.y));
      }
    }
    __syncthreads();
    double2* tmp = a; a = b; b = tmp;
    Ns *= R;
  }
  return a;
}

// nb interleaved complex FFTs of length p.n: element e of sequence c at a[e * nb + c] (the
// layout of a tile of nb adjacent columns).  Same passes as cfft_smem_t; threads stride over
// (butterfly, sequence) pairs so consecutive threads touch consecutive sequences.
template <int SIGN>
static __device__ __noinline__ double2* cfft_smem_batch(double2* a, double2* b, const FFTPlan p,
                                                        const double2* __restrict__ WM, int nb) {
  const int n = p.n;
  const int tid = threadIdx.x, nt = blockDim.x;
  int Ns = 1;
  for (int pass = 0; pass < p.nrad; ++pass) {
    const int R = p.rad[pass];
    const int nbf = n / R;
    const int tstep = n / (Ns * R);
    for (int idx = tid; idx < nbf * nb; idx += nt) {
      const int j = idx / nb, c = idx - j * nb;
      const int k = j % Ns;
      const int base = (j - k) * R + k;
      auto A = [&](int e) -> double2 { return a[e * nb + c]; };
      auto Bw = [&](int e, double2 v) { b[e * nb + c] = v; };
      if (R == 4) {
        double2 v0 = A(j), v1 = A(j + nbf), v2 = A(j + 2 * nbf), v3 = A(j + 3 * nbf);
        if (k) {
          v1 = cmul(v1, twL<SIGN>(WM, k * tstep));
          v2 = cmul(v2, twL<SIGN>(WM, 2 * k * tstep));
          v3 = cmul(v3, twL<SIGN>(WM, 3 * k * tstep));
        }
        const double2 t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3);
        const double2 t3 = rot<SIGN>(csub(v1, v3));
        Bw(base, cadd(t0, t2));
        Bw(base + Ns, cadd(t1, t3));
        Bw(base + 2 * Ns, csub(t0, t2));
        Bw(base + 3 * Ns, csub(t1, t3));
      } else if (R == 2) {
        double2 v0 = A(j), v1 = A(j + nbf);
        if (k) v1 = cmul(v1, twL<SIGN>(WM, k * tstep));
        Bw(base, cadd(v0, v1));
        Bw(base + Ns, csub(v0, v1));
      } else {
        double2 v0 = A(j), v1 = A(j + nbf), v2 = A(j + 2 * nbf);
        if (k) {
          v1 = cmul(v1, twL<SIGN>(WM, k * tstep));
          v2 = cmul(v2, twL<SIGN>(WM, 2 * k * tstep));
        }
        const double h = 0.86602540378443864676;
        const double2 t = cadd(v1, v2);
        const double2 m = make_double2(fma(-0.5, t.x, v0.x), fma(-0.5, t.y, v0.y));
        const double2 r = rot<SIGN>(csub(v1, v2));
        Bw(base, cadd(v0, t));
        Bw(base + Ns, make_double2(fma(h, r.x, m.x), fma(h, r.y, m.y)));
        Bw(base + 2 * Ns, make_double2(fma(-h, r.x, m.x), fma(-h, r.y, m.y)));
      }
    }
    __syncthreads();
    double2* tmp = a; a = b; b = tmp;
    Ns *= R;
  }
  return a;
}

__device__ __forceinline__ double2* cfft_smem(double2* a, double2* b, const FFTPlan p, const double2* __restrict__ WM,
                                              int sign) {
  return sign > 0 ? cfft_smem_t<1>(a, b, p, WM) : cfft_smem_t<-1>(a, b, p, WM);
}


// ---- real transforms on the packed half-length sequence ---------------------------------
//
// c2r: coefficients c_k (k < K, read through get(k)) of a real field, g_j = sum over the
// Hermitian-completed spectrum with weights w0 (k = 0, real part only) and w (k >= 1):
//   g_j = w0 Re c_0 + w * 2 Re sum_{k=1}^{K-1} c_k e^{2 pi i k j / M}
// Fills Z (length L) so that the inverse L-point FFT of Z is z_j = g_{2j} + i g_{2j+1}.
template <bool UNIT, class Get>
__device__ __forceinline__ void c2r_pre_t(double2* Z, Get get, int K, int L, const double2* __restrict__ WM,
                                          double w0, double w) {
  for (int k = threadIdx.x; k < L; k += blockDim.x) {
    double2 xk = make_double2(0.0, 0.0), xc = make_double2(0.0, 0.0);
    if (k == 0) {
      xk = make_double2(UNIT ? get(0).x : w0 * get(0).x, 0.0);
    } else if (k < K) {
      xk = UNIT ? get(k) : cscale(get(k), w);
    }
    const int kc = L - k;  // partner index (k = 0 pairs with the unstored Nyquist L)
    if (k > 0 && kc < K) xc = cconj(UNIT ? get(kc) : cscale(get(kc), w));
    Z[k] = c2r_combine(cadd(xk, xc), csub(xk, xc), __ldg(&WM[k]));  // e + i (xk - xc) exp(+2 pi i k / M)
  }
}
template <class Get>
__device__ __forceinline__ void c2r_pre(double2* Z, Get get, int K, int L, const double2* __restrict__ WM,
                                        double w0, double w) {
  if (w0 == 1.0 && w == 1.0) c2r_pre_t<true>(Z, get, K, L, WM, w0, w);
  else c2r_pre_t<false>(Z, get, K, L, WM, w0, w);
}

// r2c post: z = forward L-point FFT of the packed real field; returns
//   X_k = sum_j g_j e^{-2 pi i k j / M}  for k < K  (via put(k, X_k)).
// r2c_post2: the same with put(k, 2 X_k), for callers that fold the factor 1/2 into their own
// scaling.
template <class Put>
__device__ __forceinline__ void r2c_post2(const double2* Z, Put put, int K, int L, const double2* __restrict__ WM) {
  for (int k = threadIdx.x; k < K; k += blockDim.x)
    put(k, r2c_combine2(Z[k], cconj(Z[k == 0 ? 0 : L - k]), __ldg(&WM[k])));
}
template <class Put>
__device__ __forceinline__ void r2c_post(const double2* Z, Put put, int K, int L, const double2* __restrict__ WM) {
  for (int k = threadIdx.x; k < K; k += blockDim.x)
    put(k, r2c_combine(Z[k], cconj(Z[k == 0 ? 0 : L - k]), __ldg(&WM[k])));
}

}  // namespace spadj
