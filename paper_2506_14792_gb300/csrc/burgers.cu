// 1D viscous Burgers, u_t - nu u_xx = -d/dx(u^2/2), periodic Fourier basis, 3/2 dealiasing.
//
// The whole batch runs as persistent trajectories: one CTA owns one batch member for all
// steps, keeps the multistep history (X_{n-1}, X_{n-2}, F_{n-1}, F_{n-2}) in registers and
// evaluates F through shared-memory FFTs (grid of M = 3N/2 points, one L = M/2 complex FFT
// per real transform).  Kernels:
//   * forward  -- eq. imex, SBDF<s> with s = min(n, order), order 1..4 (Supplementary A.4); M = I and
//                 L = nu k^2, so the implicit solve is a per-mode division, fused.
//   * tangent  -- the JVP of the same recurrence, run alongside the primal.
//   * adjoint  -- eq. IMEX_adjoint backward over the stored trajectory; one VJP of F per
//                 step, (dF/dX)^dagger w = B^dagger[(B X) * T^dagger(i k w)].
// State layout: [member][k] complex (k = 0..K-1), Im c_0 held at 0 after every solve.
#include <cmath>
#include <vector>

#include "fft.cuh"
#include "problem.h"

namespace spadj {
namespace {

constexpr int kQMax = 4;  // modes per thread

constexpr int kMaxOrder = 4;

struct BurgersParams {
  int K, L, M;
  double nu, kscale, dt, length;
  int order, nonlinear;
  FFTPlan plan;
  const double2* WM;
  // SBDF<s> weights, s = 1..kMaxOrder (row s-1): backward differentiation weights already divided
  // by dt (no division in the step loops) and extrapolation weights of F
  double wa[kMaxOrder][kMaxOrder + 1], wc[kMaxOrder][kMaxOrder + 1];
};

struct Smem {
  double2* A;
  double2* B;
  double2* C;
  double2* D;
  double2* S;  // spectrum staging (K)
  double2* O;  // spectral output staging (K)
};

__device__ __forceinline__ Smem carve(const BurgersParams& P) {
  extern __shared__ double2 sm[];
  Smem s;
  s.A = sm;
  s.B = s.A + P.L;
  s.C = s.B + P.L;
  s.D = s.C + P.L;
  s.S = s.D + P.L;
  s.O = s.S + P.K;
  return s;
}

// grid (packed) of the coefficients in S, weights (w0, w): see c2r_pre.  Result buffer returned.
__device__ double2* c2g_packed(const BurgersParams& P, const double2* S, double2* a, double2* b, double w0,
                               double w) {
  c2r_pre(a, [&](int k) { return S[k]; }, P.K, P.L, P.WM, w0, w);
  __syncthreads();
  return cfft_smem(a, b, P.plan, P.WM, +1);
}

// forward real FFT of the packed grid in a; writes scale(k, 2 X_k) to O (k < K): the factor 1/2
// of the real-transform unpacking is left to the scale functors.
template <class Scale>
__device__ void g2c_packed(const BurgersParams& P, double2* a, double2* b, double2* O, Scale scale) {
  double2* z = cfft_smem(a, b, P.plan, P.WM, -1);
  r2c_post2(z, [&](int k, double2 v) { O[k] = scale(k, v); }, P.K, P.L, P.WM);
  __syncthreads();
}

__device__ __forceinline__ double kwav(const BurgersParams& P, int k) { return P.kscale * k; }

// O <- F(S) = -i k T[(B S)^2 / 2]
__device__ void eval_F(const BurgersParams& P, Smem& s) {
  double2* u = c2g_packed(P, s.S, s.A, s.B, 1.0, 1.0);
  for (int j = threadIdx.x; j < P.L; j += blockDim.x) {
    double2 v = u[j];
    u[j] = make_double2(v.x * v.x, v.y * v.y);  // u^2; the 1/2 goes into the scale below
  }
  __syncthreads();
  double2* other = (u == s.A) ? s.B : s.A;
  const double q = 0.25 / P.M;  // (1/2 of u^2/2) (1/2 of the unpacking) / M
  g2c_packed(P, u, other, s.O, [&](int k, double2 v) {
    double kk = kwav(P, k) * q;  // -i k v / M
    return make_double2(kk * v.y, -kk * v.x);
  });
}

// From the primal spectrum S and the tangent spectrum S2: O <- F(S) (if want_F) and
// O2 <- (dF/dX)(S) S2 = -i k T[(B S)(B S2)].
__device__ void eval_F_and_jvp(const BurgersParams& P, Smem& s, const double2* S2, double2* O2, bool want_F) {
  // both inverse transforms in the same FFT passes (A|B and C|D are 2L apart)
  c2r_pre(s.A, [&](int k) { return s.S[k]; }, P.K, P.L, P.WM, 1.0, 1.0);
  c2r_pre(s.C, [&](int k) { return S2[k]; }, P.K, P.L, P.WM, 1.0, 1.0);
  __syncthreads();
  cfft_smem_sets<1>(s.A, s.B, 2 * P.L, 2, P.plan, 1);
  const bool odd = P.plan.nrad & 1;
  double2* u = odd ? s.B : s.A;
  double2* du = odd ? s.D : s.C;
  double2* uo = odd ? s.A : s.B;
  double2* duo = odd ? s.C : s.D;
  for (int j = threadIdx.x; j < P.L; j += blockDim.x) {
    double2 v = u[j], dv = du[j];
    du[j] = make_double2(v.x * dv.x, v.y * dv.y);
    u[j] = make_double2(v.x * v.x, v.y * v.y);
  }
  __syncthreads();
  const double qf = 0.25 / P.M, qj = 0.5 / P.M;  // -i k (u^2/2) / M and -i k (u du) / M, unpacking 1/2 included
  auto mikf = [&](int k, double2 v) {
    double kk = kwav(P, k) * qf;
    return make_double2(kk * v.y, -kk * v.x);
  };
  auto mikj = [&](int k, double2 v) {
    double kk = kwav(P, k) * qj;
    return make_double2(kk * v.y, -kk * v.x);
  };
  if (want_F) g2c_packed(P, u, uo, s.O, mikf);
  g2c_packed(P, du, duo, O2, mikj);
}

// O <- (dF/dX)(S)^dagger W  with W staged in S2:  B^dagger[(B S) * T^dagger(i k W)]
__device__ void eval_vjp(const BurgersParams& P, Smem& s, double2* S2) {
  // S2 <- i k W / (2M) (in place, own entries only): T^dagger's weights (1/M on the real part of
  // k = 0, 1/(2M) elsewhere) folded in, the k = 0 entry being 0
  const double q = 0.5 / P.M;
  for (int k = threadIdx.x; k < P.K; k += blockDim.x) {
    double2 w = S2[k];
    double kk = kwav(P, k) * q;
    S2[k] = make_double2(-kk * w.y, kk * w.x);
  }
  __syncthreads();
  // both inverse transforms in the same FFT passes (A|B and C|D are 2L apart)
  c2r_pre(s.A, [&](int k) { return s.S[k]; }, P.K, P.L, P.WM, 1.0, 1.0);
  c2r_pre(s.C, [&](int k) { return S2[k]; }, P.K, P.L, P.WM, 1.0, 1.0);
  __syncthreads();
  cfft_smem_sets<1>(s.A, s.B, 2 * P.L, 2, P.plan, 1);
  const bool odd = P.plan.nrad & 1;
  double2* u = odd ? s.B : s.A;
  double2* v = odd ? s.D : s.C;
  double2* vo = odd ? s.C : s.D;
  for (int j = threadIdx.x; j < P.L; j += blockDim.x) {
    double2 a = u[j], b = v[j];
    v[j] = make_double2(a.x * b.x, a.y * b.y);
  }
  __syncthreads();
  g2c_packed(P, v, vo, s.O, [&](int k, double2 x) {  // x = 2 X_k
    return k == 0 ? make_double2(0.5 * x.x, 0.0) : x;
  });
}

__device__ __forceinline__ const double2* row(const double* base, int b, int K) {
  return reinterpret_cast<const double2*>(base) + (size_t)b * K;
}
__device__ __forceinline__ double2* row(double* base, int b, int K) {
  return reinterpret_cast<double2*>(base) + (size_t)b * K;
}

// ---- single-shot kernels (transforms, F, JVP, VJP) ----------------------------------------

__global__ void transform_kernel(BurgersParams P, int kind, const double* __restrict__ in, double* __restrict__ out) {
  Smem s = carve(P);
  const int b = blockIdx.x;
  const int K = P.K, L = P.L, M = P.M;
  if (kind == 0 || kind == 3) {  // coefficients -> grid
    const double2* x = row(in, b, K);
    for (int k = threadIdx.x; k < K; k += blockDim.x) s.S[k] = x[k];
    __syncthreads();
    double2* z = (kind == 0) ? c2g_packed(P, s.S, s.A, s.B, 1.0, 1.0)
                             : c2g_packed(P, s.S, s.A, s.B, 1.0 / M, 0.5 / M);
    double2* g = reinterpret_cast<double2*>(out + (size_t)b * M);
    for (int j = threadIdx.x; j < L; j += blockDim.x) g[j] = z[j];
  } else {  // grid -> coefficients
    const double2* g = reinterpret_cast<const double2*>(in + (size_t)b * M);
    for (int j = threadIdx.x; j < L; j += blockDim.x) s.A[j] = g[j];
    __syncthreads();
    double2* y = row(out, b, K);
    if (kind == 1) {
      const double halfinvM = 0.5 / M;
      g2c_packed(P, s.A, s.B, s.O, [&](int k, double2 v) { return cscale(v, halfinvM); });
    } else {
      g2c_packed(P, s.A, s.B, s.O, [&](int k, double2 v) {
        return k == 0 ? make_double2(0.5 * v.x, 0.0) : v;
      });
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) y[k] = s.O[k];
  }
}

__global__ void F_kernel(BurgersParams P, int mode, const double* __restrict__ x, const double* __restrict__ d,
                         double* __restrict__ out) {
  Smem s = carve(P);
  extern __shared__ double2 sm[];
  double2* S2 = sm + 4 * P.L + 2 * P.K;  // second input spectrum (JVP direction / VJP cotangent)
  double2* O2 = S2 + P.K;                // second output spectrum
  const int b = blockIdx.x, K = P.K;
  const double2* xr = row(x, b, K);
  double2* o = row(out, b, K);
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    s.S[k] = xr[k];
    if (mode != 0) S2[k] = row(d, b, K)[k];
  }
  __syncthreads();
  if (!P.nonlinear) {
    for (int k = threadIdx.x; k < K; k += blockDim.x) o[k] = make_double2(0.0, 0.0);
    return;
  }
  if (mode == 0) {
    eval_F(P, s);
    for (int k = threadIdx.x; k < K; k += blockDim.x) o[k] = s.O[k];
  } else if (mode == 1) {
    eval_F_and_jvp(P, s, S2, O2, false);
    for (int k = threadIdx.x; k < K; k += blockDim.x) o[k] = O2[k];
  } else {
    eval_vjp(P, s, S2);
    for (int k = threadIdx.x; k < K; k += blockDim.x) o[k] = s.O[k];
  }
}

// ---- persistent trajectory kernels ----------------------------------------------------------

// Weights of step n (eq. imex with M = I, b_0 = 1, b_i = 0): SBDF<s>, s = min(n, order) (the
// scheme starts at lower order while fewer past steps exist).  a: backward differentiation
// weights (divided by dt), c: extrapolation weights of F; entries beyond s are zero.
struct Coef {
  double a[kMaxOrder + 1], c[kMaxOrder + 1];
};
constexpr double kSbdfA[kMaxOrder][kMaxOrder + 1] = {{1.0, -1.0, 0.0, 0.0, 0.0},
                                                     {1.5, -2.0, 0.5, 0.0, 0.0},
                                                     {11.0 / 6.0, -3.0, 1.5, -1.0 / 3.0, 0.0},
                                                     {25.0 / 12.0, -4.0, 3.0, -4.0 / 3.0, 0.25}};
constexpr double kSbdfC[kMaxOrder][kMaxOrder + 1] = {{0.0, 1.0, 0.0, 0.0, 0.0},
                                                     {0.0, 2.0, -1.0, 0.0, 0.0},
                                                     {0.0, 3.0, -3.0, 1.0, 0.0},
                                                     {0.0, 4.0, -6.0, 4.0, -1.0}};
__device__ __forceinline__ int step_order(const BurgersParams& P, int n) { return n < P.order ? n : P.order; }
__device__ __forceinline__ Coef step_coef(const BurgersParams& P, int n) {
  Coef c;
  const int s = step_order(P, n);
#pragma unroll
  for (int i = 0; i <= kMaxOrder; ++i) {
    c.a[i] = P.wa[s - 1][i];
    c.c[i] = P.wc[s - 1][i];
  }
  return c;
}
__device__ __forceinline__ Coef zero_coef() {
  Coef c;
#pragma unroll
  for (int i = 0; i <= kMaxOrder; ++i) c.a[i] = c.c[i] = 0.0;
  return c;
}

__device__ __forceinline__ double2 axpby(double a, double2 x, double b, double2 y) {
  return make_double2(fma(a, x.x, b * y.x), fma(a, x.y, b * y.y));
}

// sum over the history terms i = 2..ORD of c_i H_F[i-1] - a_i H_X[i-1] added to r (the i = 1
// term starts r); terms whose weights are zero add nothing
template <int ORD>
__device__ __forceinline__ double2 hist_rhs(const Coef& c, const double2 (&hf)[ORD], const double2 (&hx)[ORD]) {
  double2 r = axpby(c.c[1], hf[0], -c.a[1], hx[0]);
#pragma unroll
  for (int i = 2; i <= ORD; ++i)
    if (c.c[i] != 0.0 || c.a[i] != 0.0)
      r = make_double2(r.x + c.c[i] * hf[i - 1].x - c.a[i] * hx[i - 1].x,
                       r.y + c.c[i] * hf[i - 1].y - c.a[i] * hx[i - 1].y);
  return r;
}

// mode 0: forward (optionally storing traj), mode 1: tangent.  ORD = the history length kept
// in registers (2 for SBDF1/2, 4 for SBDF3/4): X_{n-1..n-ORD}, F_{n-1..n-ORD} (and their tangents).
template <int Q, int ORD>
__global__ void __launch_bounds__(64) trajectory_kernel(BurgersParams P, int n_steps, const double* __restrict__ x0,
                                                        const double* __restrict__ dx0, double* __restrict__ x_out,
                                                        double* __restrict__ traj, int tangent) {
  Smem s = carve(P);
  extern __shared__ double2 sm[];
  double2* S2 = sm + 4 * P.L + 2 * P.K;
  double2* O2 = S2 + P.K;
  const int b = blockIdx.x, K = P.K, G = blockDim.x, tid = threadIdx.x;
  const int nb = gridDim.x;
  double2 X[Q][ORD], F[Q][ORD], D[Q][ORD], GJ[Q][ORD];
  const double2* xr = row(x0, b, K);
  for (int q = 0; q < Q; ++q) {
    int k = tid + q * G;
    double2 z = make_double2(0.0, 0.0);
#pragma unroll
    for (int i = 0; i < ORD; ++i) X[q][i] = F[q][i] = D[q][i] = GJ[q][i] = z;
    X[q][0] = (k < K) ? xr[k] : z;
    if (tangent && k < K) D[q][0] = row(dx0, b, K)[k];
    if (k < K) {
      s.S[k] = X[q][0];
      if (tangent) S2[k] = D[q][0];
      if (traj) row(traj, b, K)[k] = X[q][0];
    }
  }
  __syncthreads();
  if (P.nonlinear) {
    if (tangent) eval_F_and_jvp(P, s, S2, O2, true);
    else eval_F(P, s);
    for (int q = 0; q < Q; ++q) {
      int k = tid + q * G;
      if (k < K) { F[q][0] = s.O[k]; if (tangent) GJ[q][0] = O2[k]; }
    }
  }
  // nu k^2 per mode and 1 / (a_0 + nu k^2), recomputed only when the step order changes
  double nk2[Q], inv_m[Q];
  for (int q = 0; q < Q; ++q) {
    const double kk = kwav(P, tid + q * G);
    nk2[q] = P.nu * kk * kk;
    inv_m[q] = 0.0;
  }
  int s_prev = 0;
  for (int n = 1; n <= n_steps; ++n) {
    Coef c = step_coef(P, n);
    const int s_n = step_order(P, n);
    if (s_n != s_prev) {
      for (int q = 0; q < Q; ++q) inv_m[q] = 1.0 / (c.a[0] + nk2[q]);
      s_prev = s_n;
    }
    for (int q = 0; q < Q; ++q) {
      int k = tid + q * G;
      if (k >= K) continue;
      const double inv = inv_m[q];
      double2 xn = cscale(hist_rhs<ORD>(c, F[q], X[q]), inv);
      if (k == 0) xn.y = 0.0;
#pragma unroll
      for (int i = ORD - 1; i > 0; --i) { X[q][i] = X[q][i - 1]; F[q][i] = F[q][i - 1]; }
      X[q][0] = xn;
      s.S[k] = xn;
      if (traj) row(traj + (size_t)n * nb * 2 * K, b, K)[k] = xn;
      if (tangent) {
        double2 dn = cscale(hist_rhs<ORD>(c, GJ[q], D[q]), inv);
        if (k == 0) dn.y = 0.0;
#pragma unroll
        for (int i = ORD - 1; i > 0; --i) { D[q][i] = D[q][i - 1]; GJ[q][i] = GJ[q][i - 1]; }
        D[q][0] = dn;
        S2[k] = dn;
      }
    }
    __syncthreads();
    if (n < n_steps && P.nonlinear) {
      if (tangent) eval_F_and_jvp(P, s, S2, O2, true);
      else eval_F(P, s);
      for (int q = 0; q < Q; ++q) {
        int k = tid + q * G;
        if (k < K) { F[q][0] = s.O[k]; if (tangent) GJ[q][0] = O2[k]; }
      }
    }
  }
  double2* o = row(x_out, b, K);
  for (int q = 0; q < Q; ++q) {
    int k = tid + q * G;
    if (k < K) o[k] = tangent ? D[q][0] : X[q][0];
  }
}

// Adjoint sweep (eq. IMEX_adjoint) over traj = X_0..X_N, seeded by y_final = dJ/dX_N.
// seed_at (nullable, device, n_steps+1 ints): index into seeds ([n][member][k]) of the
// cotangent injected at X_n, or -1; when seed_at is NULL the only seed is y_final at X_N.
template <int Q, int ORD>
__global__ void __launch_bounds__(64) adjoint_kernel(BurgersParams P, int n_steps, const double* __restrict__ traj,
                                                     const double* __restrict__ y_final, double* __restrict__ grad,
                                                     const int* __restrict__ seed_at, const double* __restrict__ seeds) {
  Smem s = carve(P);
  extern __shared__ double2 sm[];
  double2* S2 = sm + 4 * P.L + 2 * P.K;
  const int b = blockIdx.x, K = P.K, G = blockDim.x, tid = threadIdx.x;
  const int nb = gridDim.x;
  const size_t stride = (size_t)nb * 2 * K;
  double2 Y[Q][ORD];  // Y_{n+1}, ..., Y_{n+ORD}
  const double2 z = make_double2(0.0, 0.0);
  // nu k^2 per mode and 1 / (a_0 + nu k^2) of the current step order (steps run backward, so the
  // order changes only over the first steps)
  double nk2[Q], inv_m[Q];
  for (int q = 0; q < Q; ++q) {
    const double kk = kwav(P, tid + q * G);
    nk2[q] = P.nu * kk * kk;
    inv_m[q] = 0.0;
  }
  int s_prev = 0;
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int i = 0; i < ORD; ++i) Y[q][i] = z;
  for (int n = n_steps; n >= 0; --n) {
    double2 lam[Q];
    if (n == n_steps) {
      for (int q = 0; q < Q; ++q) {
        int k = tid + q * G;
        lam[q] = (k < K && y_final) ? row(y_final, b, K)[k] : z;
      }
    } else {
      // the weights of step n+i that multiply X_n: c_i^{n+i}, a_i^{n+i} (zero past the horizon)
      double wc[ORD + 1], wa[ORD + 1];
#pragma unroll
      for (int i = 1; i <= ORD; ++i) {
        const Coef ci = (n + i <= n_steps) ? step_coef(P, n + i) : zero_coef();
        wc[i] = ci.c[i];
        wa[i] = ci.a[i];
      }
      const double2* xn = row(traj + (size_t)n * stride, b, K);
      for (int q = 0; q < Q; ++q) {
        int k = tid + q * G;
        if (k >= K) continue;
        s.S[k] = xn[k];
        double2 w = axpby(wc[1], Y[q][0], wc[2], Y[q][1]);
#pragma unroll
        for (int i = 3; i <= ORD; ++i) w = make_double2(w.x + wc[i] * Y[q][i - 1].x, w.y + wc[i] * Y[q][i - 1].y);
        S2[k] = w;
      }
      __syncthreads();
      if (P.nonlinear) eval_vjp(P, s, S2);
      for (int q = 0; q < Q; ++q) {
        int k = tid + q * G;
        if (k >= K) { lam[q] = z; continue; }
        double2 v = P.nonlinear ? s.O[k] : z;
        double2 l = make_double2(v.x - wa[1] * Y[q][0].x - wa[2] * Y[q][1].x, v.y - wa[1] * Y[q][0].y - wa[2] * Y[q][1].y);
#pragma unroll
        for (int i = 3; i <= ORD; ++i) l = make_double2(l.x - wa[i] * Y[q][i - 1].x, l.y - wa[i] * Y[q][i - 1].y);
        lam[q] = l;
      }
      __syncthreads();
    }
    if (seed_at && seed_at[n] >= 0) {
      const double* sv = seeds + (size_t)seed_at[n] * nb * 2 * K;
      for (int q = 0; q < Q; ++q) {
        int k = tid + q * G;
        if (k < K) lam[q] = cadd(lam[q], row(sv, b, K)[k]);
      }
    }
    if (n == 0) {
      double2* g = row(grad, b, K);
      for (int q = 0; q < Q; ++q) {
        int k = tid + q * G;
        if (k < K) g[k] = lam[q];
      }
      return;
    }
    const int s_n = step_order(P, n);
    if (s_n != s_prev) {
      const Coef c = step_coef(P, n);
      for (int q = 0; q < Q; ++q) inv_m[q] = 1.0 / (c.a[0] + nk2[q]);
      s_prev = s_n;
    }
    for (int q = 0; q < Q; ++q) {
      int k = tid + q * G;
      if (k >= K) continue;
      double2 y = cscale(lam[q], inv_m[q]);
      if (k == 0) y.y = 0.0;
#pragma unroll
      for (int i = ORD - 1; i > 0; --i) Y[q][i] = Y[q][i - 1];
      Y[q][0] = y;
    }
  }
}

// J_b = (length/2)(Re c_0^2 + 2 sum_{k>=1} |c_k|^2) and seed y = dJ/dX.
__global__ void energy_kernel(BurgersParams P, const double* __restrict__ x, double* __restrict__ J,
                              double* __restrict__ seed) {
  const int b = blockIdx.x, K = P.K;
  const double2* xr = row(x, b, K);
  double2* y = row(seed, b, K);
  double acc = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double2 v = xr[k];
    if (k == 0) {
      acc += v.x * v.x;
      y[k] = make_double2(P.length * v.x, 0.0);
    } else {
      acc += 2.0 * (v.x * v.x + v.y * v.y);
      y[k] = make_double2(2.0 * P.length * v.x, 2.0 * P.length * v.y);
    }
  }
  __shared__ double red[128];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) J[b] = 0.5 * P.length * red[0];
}

// ---- host side --------------------------------------------------------------------------------

struct Burgers : EqImpl {
  BurgersParams P{};
  int B = 1;
  int G = 64;
  DevBuf wm, traj, seed, Jd;
  size_t smem = 0;

  size_t state_len(int which) const override {
    if (which == 0) return (size_t)B * 2 * P.K;
    if (which == 1) return (size_t)B * P.M;
    if (which == 3) return (size_t)B * 2 * P.K;
    return 0;
  }

  spadj_status init(Problem* p) {
    const spadj_desc& d = p->desc;
    if (d.n[0] < 4 || d.n[0] % 4 != 0) return p->fail(SPADJ_ERR_INVALID, "burgers: n[0] must be a positive multiple of 4");
    B = d.batch;
    P.K = d.n[0] / 2;
    P.M = 3 * d.n[0] / 2;
    P.L = P.M / 2;
    P.length = d.length[0] > 0 ? d.length[0] : 2.0 * M_PI;
    P.kscale = 2.0 * M_PI / P.length;
    P.nu = d.params[0];
    P.dt = d.dt;
    switch (d.scheme) {
      case SPADJ_SBDF1: P.order = 1; break;
      case SPADJ_SBDF2: P.order = 2; break;
      case SPADJ_SBDF3: P.order = 3; break;
      case SPADJ_SBDF4: P.order = 4; break;
      default: return p->fail(SPADJ_ERR_UNSUPPORTED, "burgers: scheme must be SBDF1, SBDF2, SBDF3 or SBDF4");
    }
    P.nonlinear = d.nonlinear;
    for (int s = 0; s < kMaxOrder; ++s)
      for (int i = 0; i <= kMaxOrder; ++i) {
        P.wa[s][i] = kSbdfA[s][i] / P.dt;
        P.wc[s][i] = kSbdfC[s][i];
      }
    P.plan = make_plan(P.L);
    if (P.plan.nrad < 0) return p->fail(SPADJ_ERR_INVALID, "burgers: 3N/4 must be of the form 2^a 3^b");
    if (P.K > kQMax * G) return p->fail(SPADJ_ERR_INVALID, "burgers: n[0] too large (max 512)");
    std::vector<double2> h(P.M);
    for (int m = 0; m < P.M; ++m) {
      double th = -2.0 * M_PI * (double)m / (double)P.M;
      h[m] = make_double2(std::cos(th), std::sin(th));
    }
    {  // the butterflies' scaled-twiddle records follow the M-table in the same buffer
      const std::vector<double2> sct = scaled_twiddle_table(P.plan);
      h.insert(h.end(), sct.begin(), sct.end());
    }
    SPADJ_CUDA_TRY(p, wm.ensure(sizeof(double2) * h.size()));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(wm.ptr, h.data(), sizeof(double2) * h.size(), cudaMemcpyHostToDevice, p->stream));
    SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    P.WM = wm.as<double2>();
    bind_scaled_twiddles(P.plan, P.WM + P.M);
    smem = sizeof(double2) * (4 * P.L + 4 * P.K);
    return SPADJ_OK;
  }

  spadj_status transform(Problem* p, int kind, const double* in, double* out) override {
    if (kind < 0 || kind > 3) return p->fail(SPADJ_ERR_INVALID, "transform: kind must be 0..3");
    transform_kernel<<<B, G, smem, p->stream>>>(P, kind, in, out);
    return check_launch(p, "burgers transform");
  }

  spadj_status eval_F(Problem* p, int mode, const double* x, const double* dx, double* out) override {
    F_kernel<<<B, G, smem, p->stream>>>(P, mode, x, dx, out);
    return check_launch(p, "burgers F");
  }

  // modes per thread Q and register history length (2 for SBDF1/2, 4 for SBDF3/4)
  template <class Fn>
  spadj_status dispatchQ(Problem* p, Fn fn) {
    int Q = (P.K + G - 1) / G;
    auto byQ = [&](auto ord) {
      if (Q <= 1) fn(std::integral_constant<int, 1>(), ord);
      else if (Q == 2) fn(std::integral_constant<int, 2>(), ord);
      else fn(std::integral_constant<int, 4>(), ord);
    };
    if (P.order <= 2) byQ(std::integral_constant<int, 2>());
    else byQ(std::integral_constant<int, 4>());
    return check_launch(p, "burgers trajectory");
  }

  // algorithmic FP64 flops per member-step: real FFTs of M points (2.5 M log2 M each) plus
  // the pointwise product and the per-mode combine.
  double fft_flops() const { return 2.5 * P.M * std::log2((double)P.M); }

  spadj_status forward(Problem* p, int n_steps, const double* x0, double* x_out, double* trj) override {
    if (n_steps < 0) return p->fail(SPADJ_ERR_INVALID, "forward: n_steps < 0");
    cudaEvent_t t = p->tic();
    spadj_status s = dispatchQ(p, [&](auto q, auto o) {
      trajectory_kernel<decltype(q)::value, decltype(o)::value><<<B, G, smem, p->stream>>>(P, n_steps, x0, nullptr,
                                                                                         x_out, trj, 0);
    });
    p->toc(t, KC_FUSED, (double)B * n_steps * (2 * fft_flops() + P.M + 10.0 * P.K));
    return s;
  }

  spadj_status tangent(Problem* p, int n_steps, const double* x0, const double* dx0, double* dx_out) override {
    if (n_steps < 0) return p->fail(SPADJ_ERR_INVALID, "tangent: n_steps < 0");
    return dispatchQ(p, [&](auto q, auto o) {
      trajectory_kernel<decltype(q)::value, decltype(o)::value><<<B, G, smem, p->stream>>>(P, n_steps, x0, dx0, dx_out,
                                                                                         nullptr, 1);
    });
  }

  const int* seed_dev = nullptr;     // set only during vjp()
  const double* seeds_dev = nullptr;
  DevBuf seedmap;

  spadj_status vjp(Problem* p, const double* x0, int n_steps, int ckpt_slots, const std::vector<int>& seed_at,
                   const double* seeds, double* grad) override {
    (void)ckpt_slots;  // the per-member persistent kernels keep the whole trajectory (store-all)
    if (n_steps < 1) return p->fail(SPADJ_ERR_INVALID, "vjp: n_steps < 1");
    const size_t sl = state_len(0);
    SPADJ_CUDA_TRY(p, traj.ensure(sizeof(double) * sl * (size_t)(n_steps + 1)));
    SPADJ_CUDA_TRY(p, seedmap.ensure(sizeof(int) * (size_t)(n_steps + 1)));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(seedmap.ptr, seed_at.data(), sizeof(int) * (n_steps + 1), cudaMemcpyHostToDevice,
                                      p->stream));
    double* T = traj.as<double>();
    spadj_status st = forward(p, n_steps, x0, T + (size_t)n_steps * sl, T);
    if (st != SPADJ_OK) return st;
    seed_dev = seedmap.as<int>();
    seeds_dev = seeds;
    st = adjoint(p, n_steps, T, nullptr, grad);
    seed_dev = nullptr;
    seeds_dev = nullptr;
    if (st != SPADJ_OK) return st;
    SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));  // seed_at host staging is pageable
    return SPADJ_OK;
  }

  spadj_status adjoint(Problem* p, int n_steps, const double* trj, const double* y_final, double* grad) override {
    if (n_steps < 1) return p->fail(SPADJ_ERR_INVALID, "adjoint: n_steps < 1");
    cudaEvent_t t = p->tic();
    spadj_status s = dispatchQ(p, [&](auto q, auto o) {
      adjoint_kernel<decltype(q)::value, decltype(o)::value><<<B, G, smem, p->stream>>>(P, n_steps, trj, y_final, grad,
                                                                                      seed_dev, seeds_dev);
    });
    p->toc(t, KC_FUSED, (double)B * n_steps * (3 * fft_flops() + 2.0 * P.M + 12.0 * P.K));
    return s;
  }

  spadj_status objective(Problem* p, int objective, const double* obj_data, const double* x, double* J_dev,
                         double* sd) override {
    (void)obj_data;
    if (objective != SPADJ_OBJ_ENERGY) return p->fail(SPADJ_ERR_UNSUPPORTED, "burgers: objective must be ENERGY");
    energy_kernel<<<B, 128, 0, p->stream>>>(P, x, J_dev, sd);
    return check_launch(p, "burgers energy");
  }

  spadj_status gradient(Problem* p, const double* x0, int n_steps, int objective, const double* obj_data,
                        int ckpt_slots, double* J_host, double* grad, double* grad_p) override {
    (void)obj_data; (void)ckpt_slots; (void)grad_p;
    if (objective != SPADJ_OBJ_ENERGY) return p->fail(SPADJ_ERR_UNSUPPORTED, "burgers: objective must be ENERGY");
    if (n_steps < 1) return p->fail(SPADJ_ERR_INVALID, "gradient: n_steps < 1");
    const size_t sl = state_len(0);
    SPADJ_CUDA_TRY(p, traj.ensure(sizeof(double) * sl * (size_t)(n_steps + 1)));
    SPADJ_CUDA_TRY(p, seed.ensure(sizeof(double) * sl));
    SPADJ_CUDA_TRY(p, Jd.ensure(sizeof(double) * B));
    double* T = traj.as<double>();
    double* xN = T + (size_t)n_steps * sl;
    spadj_status st = forward(p, n_steps, x0, xN, T);
    if (st != SPADJ_OK) return st;
    if ((st = this->objective(p, objective, obj_data, xN, Jd.as<double>(), seed.as<double>())) != SPADJ_OK) return st;
    st = adjoint(p, n_steps, T, seed.as<double>(), grad);
    if (st != SPADJ_OK) return st;
    if (J_host) {
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(J_host, Jd.ptr, sizeof(double) * B, cudaMemcpyDeviceToHost, p->stream));
      SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
      for (int i = 0; i < B; ++i)
        if (!std::isfinite(J_host[i])) return p->fail(SPADJ_ERR_NONFINITE, "burgers: objective is not finite");
    }
    return SPADJ_OK;
  }

  ~Burgers() override {
    wm.release();
    seedmap.release();
    traj.release();
    seed.release();
    Jd.release();
  }
};

}  // namespace

EqImpl* make_burgers(Problem* p, spadj_status* st) {
  Burgers* b = new Burgers();
  *st = b->init(p);
  if (*st != SPADJ_OK) {
    delete b;
    return nullptr;
  }
  return b;
}

}  // namespace spadj
