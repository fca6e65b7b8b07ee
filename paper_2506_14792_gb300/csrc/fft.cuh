// FP64 shared-memory FFTs for the collocation transforms (Methods, "Spectral transforms").
//
// A real field of M = 2L grid points is transformed through one complex FFT of length
// L on the packed sequence z_j = g_{2j} + i g_{2j+1} (the classic half-length real FFT),
// so a 3/2-dealiased grid of 384 points costs one 192-point complex FFT.  The complex
// FFT is a Stockham autosort (ping-pong between two shared buffers, natural order in
// and out) with radix-4/3/2 passes; all threads of the CTA take part and every pass
// ends with a CTA barrier.  The real pre/post-processing takes its twiddles from a device table
//   WM[m] = exp(-2 pi i m / M),  m = 0..M-1;
// the twiddled butterflies take theirs from the plan's scaled-twiddle records (below).
//
// Scaled twiddles (the multiply-add butterflies of S. Goedecker, SIAM J. Sci. Comput. 18 (1997)
// 1605): a twiddle w = c + i s acts on v as
//   w v = lambda (v + tau i v),  lambda = c,   tau = s / c    where |c| >= |s|,
//                                lambda = i s, tau = -c / s   otherwise,
// so |tau| <= 1 and lambda is real or imaginary.  q = v + tau i v is two multiply-adds, and a
// real-or-imaginary coefficient folds into the multiply-add that applies it (an imaginary one
// swaps the components and carries the sign in its per-component scales; no FP64 instruction).
// With the ratios of the lambdas precomputed, a twiddled radix-4 butterfly takes 22 FP64
// instructions (28 with complex products), radix-3 16 (20) and radix-2 6 (8): the FP64 pipe
// is the binding resource of every transform here.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

namespace spadj {

struct FFTPlan {
  int n;                  // complex length L
  int nrad;               // number of passes
  unsigned char rad[8];   // radix of each pass (product = n)
  const double2* sc[2];   // device scaled-twiddle records: [0] exp(-), [1] exp(+)
};

// double2 entries of one record (one twiddle index k of a pass) for radix R
__host__ __device__ constexpr int sc_rec(int R) { return R == 2 ? 2 : 6; }
// double2 entries of a pass's records (Ns = product of the earlier radices; none for Ns = 1);
// a pass's records start after those of the earlier passes
__host__ __device__ constexpr int sc_pass_entries(int R, int Ns) { return Ns > 1 ? Ns * sc_rec(R) : 0; }

// Factor n = 2^a 3^b into radix-4 passes, then one radix-2 if a is odd, then radix-3; nrad = -1
// for any other n and for more than 8 passes.
inline FFTPlan make_plan(int n) {
  FFTPlan p{};
  p.n = n;
  int m = n;
  auto push = [&](int r) {
    if (p.nrad >= 8) return false;
    p.rad[p.nrad++] = (unsigned char)r;
    m /= r;
    return true;
  };
  bool ok = n >= 1;
  while (ok && m % 4 == 0) ok = push(4);
  if (ok && m % 2 == 0) ok = push(2);
  while (ok && m % 3 == 0) ok = push(3);
  if (!ok || m != 1) p.nrad = -1;  // unsupported length
  return p;
}

// ---- host: scaled-twiddle records ---------------------------------------------------------
//
// Record of pass (R, Ns) and index k, for the twiddles w_m = exp(SIGN 2 pi i m k / (R Ns)) with
// forms (lambda_m, tau_m); a real-or-imaginary coefficient is stored as its per-component
// scales (r, r) (real r) or (-r, r) (imaginary i r, applied to the swapped components), and
// a flag word (an int64 in a double slot) says which are imaginary:
//   radix 4: (tau1, tau2) (tau3, flags) lambda2 rho=lambda3/lambda1 lambda1 kappa=SIGN i lambda1
//   radix 3: (tau1, tau2) rho=lambda2/lambda1 lambda1 -lambda1/2 kappa=(sqrt3/2) SIGN i lambda1
//            (flags, 0)
//   radix 2: (tau1, flags) lambda1
// flags: bit 0 lambda2, bit 1 rho, bit 2 lambda1 imaginary (kappa is then real).  Passes with
// Ns = 1 have no twiddles and no records.
struct ScCoef {
  bool im;
  double r;
};
inline ScCoef sc_form(double c, double s, double* tau) {
  if (std::fabs(c) >= std::fabs(s)) { *tau = s / c; return {false, c}; }
  *tau = -c / s;
  return {true, s};
}
inline ScCoef sc_div(ScCoef a, ScCoef b) {  // a / b
  if (a.im == b.im) return {false, a.r / b.r};
  return a.im ? ScCoef{true, a.r / b.r} : ScCoef{true, -a.r / b.r};
}
inline ScCoef sc_times_i(ScCoef a, double s) { return a.im ? ScCoef{false, -s * a.r} : ScCoef{true, s * a.r}; }
inline double2 sc_scales(ScCoef a) { return a.im ? make_double2(-a.r, a.r) : make_double2(a.r, a.r); }
inline double sc_flags(long long f) {
  double d;
  std::memcpy(&d, &f, sizeof d);
  return d;
}

// double2 entries of one direction's records
inline int scaled_twiddle_entries(const FFTPlan& p) {
  int e = 0, Ns = 1;
  for (int pass = 0; pass < p.nrad; ++pass) {
    e += sc_pass_entries(p.rad[pass], Ns);
    Ns *= p.rad[pass];
  }
  return e;
}

// Both directions' records (exp(-) first, then exp(+)), each in pass order; upload them and
// call bind_scaled_twiddles with the device copy.
inline std::vector<double2> scaled_twiddle_table(const FFTPlan& p) {
  std::vector<double2> t[2];
  const double pi = 3.14159265358979323846;
  for (int dir = 0; dir < 2; ++dir) {
    const int SIGN = dir == 0 ? -1 : 1;
    int Ns = 1;
    for (int pass = 0; pass < p.nrad; ++pass) {
      const int R = p.rad[pass];
      if (Ns > 1) {
        for (int k = 0; k < Ns; ++k) {
          ScCoef lam[4];
          double tau[4] = {0, 0, 0, 0};
          for (int m = 1; m < R; ++m) {
            const double th = SIGN * 2.0 * pi * (double)(m * k) / (double)(R * Ns);
            lam[m] = sc_form(std::cos(th), std::sin(th), &tau[m]);
          }
          std::vector<double2>& o = t[dir];
          if (R == 4) {
            const ScCoef rho = sc_div(lam[3], lam[1]), kap = sc_times_i(lam[1], SIGN);
            const long long f = (lam[2].im ? 1 : 0) | (rho.im ? 2 : 0) | (lam[1].im ? 4 : 0);
            o.push_back(make_double2(tau[1], tau[2]));
            o.push_back(make_double2(tau[3], sc_flags(f)));
            o.push_back(sc_scales(lam[2]));
            o.push_back(sc_scales(rho));
            o.push_back(sc_scales(lam[1]));
            o.push_back(sc_scales(kap));
          } else if (R == 3) {
            const ScCoef rho = sc_div(lam[2], lam[1]);
            const ScCoef half = {lam[1].im, -0.5 * lam[1].r};
            const ScCoef kap = sc_times_i(lam[1], 0.86602540378443864676 * SIGN);
            const long long f = (rho.im ? 2 : 0) | (lam[1].im ? 4 : 0);
            o.push_back(make_double2(tau[1], tau[2]));
            o.push_back(sc_scales(rho));
            o.push_back(sc_scales(lam[1]));
            o.push_back(sc_scales(half));
            o.push_back(sc_scales(kap));
            o.push_back(make_double2(sc_flags(f), 0.0));
          } else {
            const long long f = lam[1].im ? 4 : 0;
            o.push_back(make_double2(tau[1], sc_flags(f)));
            o.push_back(sc_scales(lam[1]));
          }
        }
      }
      Ns *= R;
    }
  }
  std::vector<double2> all(t[0]);
  all.insert(all.end(), t[1].begin(), t[1].end());
  if (all.empty()) all.push_back(make_double2(0.0, 0.0));  // one-pass plans: keep a valid pointer
  return all;
}
inline void bind_scaled_twiddles(FFTPlan& p, const double2* dev) {
  p.sc[0] = dev;
  p.sc[1] = dev + scaled_twiddle_entries(p);
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

// SIGN * i * a (exact: a swap and a sign change, no multiply)
template <int SIGN>
__device__ __forceinline__ double2 rot(double2 a) {
  return SIGN > 0 ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

// ---- device: butterflies ------------------------------------------------------------------

// Components swapped when the coefficient applied to them is imaginary.
__device__ __forceinline__ double2 sc_swap(double2 z, bool im) { return im ? make_double2(z.y, z.x) : z; }
// u + zeta z and u - zeta z for zeta with per-component scales a, z already swapped as zeta asks
__device__ __forceinline__ double2 sc_add(double2 u, double2 a, double2 z) {
  return make_double2(fma(a.x, z.x, u.x), fma(a.y, z.y, u.y));
}
__device__ __forceinline__ double2 sc_sub(double2 u, double2 a, double2 z) {
  return make_double2(fma(-a.x, z.x, u.x), fma(-a.y, z.y, u.y));
}
// v + tau i v
__device__ __forceinline__ double2 sc_q(double2 v, double t) { return make_double2(fma(-t, v.y, v.x), fma(t, v.x, v.y)); }
__device__ __forceinline__ long long sc_flagword(double d) { return __double_as_longlong(d); }

// Twiddled radix-4 butterfly in place (outputs in input order), record r: 22 multiply-adds.
//   A, B = v0 +- w2 v2;  lambda1 (E, F) = w1 v1 +- w3 v3;  y0, y2 = A +- lambda1 E;
//   y1, y3 = B +- SIGN i lambda1 F
__device__ __forceinline__ void sc_bfly4(double2& v0, double2& v1, double2& v2, double2& v3,
                                         const double2* __restrict__ r) {
  const double2 t12 = __ldg(r), t3f = __ldg(r + 1);
  const long long f = sc_flagword(t3f.y);
  const double2 q1 = sc_q(v1, t12.x);
  const double2 q2 = sc_swap(sc_q(v2, t12.y), f & 1);
  const double2 q3 = sc_swap(sc_q(v3, t3f.x), f & 2);
  const double2 l2 = __ldg(r + 2), rho = __ldg(r + 3), l1 = __ldg(r + 4), kap = __ldg(r + 5);
  const double2 A = sc_add(v0, l2, q2), B = sc_sub(v0, l2, q2);
  const double2 E = sc_swap(sc_add(q1, rho, q3), f & 4), F = sc_swap(sc_sub(q1, rho, q3), !(f & 4));
  v0 = sc_add(A, l1, E);
  v2 = sc_sub(A, l1, E);
  v1 = sc_add(B, kap, F);
  v3 = sc_sub(B, kap, F);
}
// Twiddled radix-3 butterfly in place, record r: 16 multiply-adds.
//   lambda1 (E, F) = w1 v1 +- w2 v2;  y0 = v0 + lambda1 E;  M = v0 - lambda1 E / 2;
//   y1, y2 = M +- (sqrt3/2) SIGN i lambda1 F
__device__ __forceinline__ void sc_bfly3(double2& v0, double2& v1, double2& v2, const double2* __restrict__ r) {
  const double2 t12 = __ldg(r);
  const long long f = sc_flagword(__ldg(&r[5].x));
  const double2 q1 = sc_q(v1, t12.x);
  const double2 q2 = sc_swap(sc_q(v2, t12.y), f & 2);
  const double2 rho = __ldg(r + 1), l1 = __ldg(r + 2), hl = __ldg(r + 3), kap = __ldg(r + 4);
  const double2 E = sc_swap(sc_add(q1, rho, q2), f & 4), F = sc_swap(sc_sub(q1, rho, q2), !(f & 4));
  const double2 M = sc_add(v0, hl, E);
  v0 = sc_add(v0, l1, E);
  v1 = sc_add(M, kap, F);
  v2 = sc_sub(M, kap, F);
}
// Twiddled radix-2 butterfly in place, record r: 6 multiply-adds.
__device__ __forceinline__ void sc_bfly2(double2& v0, double2& v1, const double2* __restrict__ r) {
  const double2 t = __ldg(r), l1 = __ldg(r + 1);
  const double2 q = sc_swap(sc_q(v1, t.x), sc_flagword(t.y) & 4);
  const double2 y0 = sc_add(v0, l1, q);
  v1 = sc_sub(v0, l1, q);
  v0 = y0;
}
// Butterflies of the first pass (Ns = 1: no twiddles).
template <int SIGN>
__device__ __forceinline__ void bfly4(double2& v0, double2& v1, double2& v2, double2& v3) {
  const double2 t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3);
  const double2 t3 = rot<SIGN>(csub(v1, v3));
  v0 = cadd(t0, t2);
  v1 = cadd(t1, t3);
  v2 = csub(t0, t2);
  v3 = csub(t1, t3);
}
template <int SIGN>
__device__ __forceinline__ void bfly3(double2& v0, double2& v1, double2& v2) {
  const double h = 0.86602540378443864676;  // sqrt(3)/2
  const double2 t = cadd(v1, v2);
  const double2 m = make_double2(fma(-0.5, t.x, v0.x), fma(-0.5, t.y, v0.y));
  const double2 r = rot<SIGN>(csub(v1, v2));  // m +- h r as multiply-adds
  v0 = cadd(v0, t);
  v1 = make_double2(fma(h, r.x, m.x), fma(h, r.y, m.y));
  v2 = make_double2(fma(-h, r.x, m.x), fma(-h, r.y, m.y));
}
__device__ __forceinline__ void bfly2(double2& v0, double2& v1) {
  const double2 y0 = cadd(v0, v1);
  v1 = csub(v0, v1);
  v0 = y0;
}

// One butterfly of a Stockham pass: R inputs through ld(e), outputs through st(e, v).
template <int SIGN, class Ld, class St>
__device__ __forceinline__ void stockham_bfly(int R, int Ns, int j, int nbf, const double2* __restrict__ rec,
                                              Ld ld, St st) {
  const int k = j % Ns;
  const int base = (j - k) * R + k;
  if (R == 4) {
    double2 v0 = ld(j), v1 = ld(j + nbf), v2 = ld(j + 2 * nbf), v3 = ld(j + 3 * nbf);
    if (Ns > 1) sc_bfly4(v0, v1, v2, v3, rec + sc_rec(4) * k);
    else bfly4<SIGN>(v0, v1, v2, v3);
    st(base, v0);
    st(base + Ns, v1);
    st(base + 2 * Ns, v2);
    st(base + 3 * Ns, v3);
  } else if (R == 2) {
    double2 v0 = ld(j), v1 = ld(j + nbf);
    if (Ns > 1) sc_bfly2(v0, v1, rec + sc_rec(2) * k);
    else bfly2(v0, v1);
    st(base, v0);
    st(base + Ns, v1);
  } else {  // R == 3
    double2 v0 = ld(j), v1 = ld(j + nbf), v2 = ld(j + 2 * nbf);
    if (Ns > 1) sc_bfly3(v0, v1, v2, rec + sc_rec(3) * k);
    else bfly3<SIGN>(v0, v1, v2);
    st(base, v0);
    st(base + Ns, v1);
    st(base + 2 * Ns, v2);
  }
}

// Complex FFT of length p.n held in buffer a (b is scratch of the same size).  SIGN = -1:
// forward exp(-), SIGN = +1: inverse exp(+) (unnormalised).  Returns the buffer holding
// the result (a or b).  All threads of the CTA must call it; it synchronises internally
// and on return the result is visible to every thread.  The WM argument is unused (the
// butterflies read the plan's scaled-twiddle records); it stays for the callers' symmetry
// with the real pre/post-processing.
template <int SIGN>
static __device__ __noinline__ double2* cfft_smem_t(double2* a, double2* b, const FFTPlan p,
                                                    const double2* __restrict__ WM) {
  const int n = p.n;
  const int tid = threadIdx.x, nt = blockDim.x;
  int Ns = 1;
  const double2* __restrict__ rec = p.sc[SIGN > 0 ? 1 : 0];
  for (int pass = 0; pass < p.nrad; ++pass) {
    const int R = p.rad[pass];
    const int nbf = n / R;
    for (int j = tid; j < nbf; j += nt)
      stockham_bfly<SIGN>(R, Ns, j, nbf, rec, [&](int e) { return a[e]; }, [&](int e, double2 v) { b[e] = v; });
    __syncthreads();
    double2* tmp = a; a = b; b = tmp;
    rec += sc_pass_entries(R, Ns);
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
  const double2* __restrict__ rec = p.sc[SIGN > 0 ? 1 : 0];
  for (int pass = 0; pass < p.nrad; ++pass) {
    const int R = p.rad[pass];
    const int nbf = n / R;
    for (int idx = tid; idx < nbf * nb; idx += nt) {
      const int j = idx / nb, c = idx - j * nb;
      stockham_bfly<SIGN>(R, Ns, j, nbf, rec, [&](int e) { return a[e * nb + c]; },
                          [&](int e, double2 v) { b[e * nb + c] = v; });
    }
    __syncthreads();
    double2* tmp = a; a = b; b = tmp;
    rec += sc_pass_entries(R, Ns);
    Ns *= R;
  }
  return a;
}

// ns sets of nb interleaved complex FFTs of length p.n (the layout of cfft_smem_batch), set s
// held in a + s * stride with scratch b + s * stride: the sets' butterflies share every pass and
// its barrier, and together fill more lanes than one set.  The results are in a (+ s * stride)
// when p.nrad is even, else in b.
template <int SIGN>
static __device__ __noinline__ void cfft_smem_sets(double2* a, double2* b, int stride, int ns, const FFTPlan p,
                                                   int nb) {
  const int n = p.n;
  const int tid = threadIdx.x, nt = blockDim.x;
  int Ns = 1;
  const double2* __restrict__ rec = p.sc[SIGN > 0 ? 1 : 0];
  for (int pass = 0; pass < p.nrad; ++pass) {
    const int R = p.rad[pass];
    const int nbf = n / R;
    const int per = nbf * nb;
    for (int idx = tid; idx < per * ns; idx += nt) {
      const int set = idx / per, i = idx - set * per;
      const int j = i / nb, c = i - j * nb;
      const double2* as = a + set * stride;
      double2* bs = b + set * stride;
      stockham_bfly<SIGN>(R, Ns, j, nbf, rec, [&](int e) { return as[e * nb + c]; },
                          [&](int e, double2 v) { bs[e * nb + c] = v; });
    }
    __syncthreads();
    double2* tmp = a; a = b; b = tmp;
    rec += sc_pass_entries(R, Ns);
    Ns *= R;
  }
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
// Entry k (< L) of the packed spectrum described below (UNIT: w0 = w = 1).
template <bool UNIT, class Get>
__device__ __forceinline__ double2 c2r_entry(Get get, int k, int K, int L, const double2* __restrict__ WM, double w0,
                                             double w) {
  double2 xk = make_double2(0.0, 0.0), xc = make_double2(0.0, 0.0);
  if (k == 0) {
    xk = make_double2(UNIT ? get(0).x : w0 * get(0).x, 0.0);
  } else if (k < K) {
    xk = UNIT ? get(k) : cscale(get(k), w);
  }
  const int kc = L - k;  // partner index (k = 0 pairs with the unstored Nyquist L)
  if (k > 0 && kc < K) xc = cconj(UNIT ? get(kc) : cscale(get(kc), w));
  return c2r_combine(cadd(xk, xc), csub(xk, xc), __ldg(&WM[k]));  // e + i (xk - xc) exp(+2 pi i k / M)
}
template <bool UNIT, class Get>
__device__ __forceinline__ void c2r_pre_t(double2* Z, Get get, int K, int L, const double2* __restrict__ WM,
                                          double w0, double w) {
  for (int k = threadIdx.x; k < L; k += blockDim.x) Z[k] = c2r_entry<UNIT>(get, k, K, L, WM, w0, w);
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
