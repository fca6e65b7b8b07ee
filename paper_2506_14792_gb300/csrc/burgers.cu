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
#include "revolve.h"

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
  // step-size schedule (nullable): weights of step n (1-based) at ws[5 (n - 1)] = a0, a1, a2, c1, c2
  // (variable-step SBDF1 / SBDF2), ws_len steps
  const double* ws;
  int ws_len;
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
  if (P.ws) {  // variable steps: the schedule's weights (zero past its end)
#pragma unroll
    for (int i = 0; i <= kMaxOrder; ++i) c.a[i] = c.c[i] = 0.0;
    if (n >= 1 && n <= P.ws_len) {
      const double* w = P.ws + (size_t)(n - 1) * 5;
      c.a[0] = w[0]; c.a[1] = w[1]; c.a[2] = w[2]; c.c[1] = w[3]; c.c[2] = w[4];
    }
    return c;
  }
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

// Forward (tangent = 0) or tangent (tangent = 1) segment of n_steps steps after step n_first,
// i.e. X_{n_first} -> X_{n_first + n_steps}.  ORD = the history length kept in registers (2 for
// SBDF1/2, 4 for SBDF3/4): X_{n-1..n-ORD}, F_{n-1..n-ORD} (and their tangents).
// Restart states (blocks of [B][K] complex): s = [X_n, ..., X_{n-s+1}, F(X_{n-1}), ..., F(X_{n-s+1})],
// s = P.order.  s_in holds in_blocks blocks: 1 (X_0 alone, a sweep from the initial state) or 2s-1
// (a full restart state); ds_in the same blocks of the tangent.  Outputs (each nullable): x_out the
// final state (or tangent), s_out the final restart state (or its tangent), traj the states
// X_{n_first}..X_{n_first+n_steps}.
template <int Q, int ORD>
__global__ void __launch_bounds__(64) trajectory_kernel(BurgersParams P, int n_first, int n_steps,
                                                        const double* __restrict__ s_in, int in_blocks,
                                                        const double* __restrict__ ds_in, double* __restrict__ x_out,
                                                        double* __restrict__ s_out, double* __restrict__ traj,
                                                        int tangent) {
  Smem s = carve(P);
  extern __shared__ double2 sm[];
  double2* S2 = sm + 4 * P.L + 2 * P.K;
  double2* O2 = S2 + P.K;
  const int b = blockIdx.x, K = P.K, G = blockDim.x, tid = threadIdx.x;
  const int nb = gridDim.x;
  const size_t blk = (size_t)nb * 2 * K;
  const int so = P.order;
  const int nx = in_blocks > 1 ? so : 1;  // X blocks present in s_in
  double2 X[Q][ORD], F[Q][ORD], D[Q][ORD], GJ[Q][ORD];
  for (int q = 0; q < Q; ++q) {
    int k = tid + q * G;
    double2 z = make_double2(0.0, 0.0);
#pragma unroll
    for (int i = 0; i < ORD; ++i) X[q][i] = F[q][i] = D[q][i] = GJ[q][i] = z;
    if (k < K) {
#pragma unroll
      for (int i = 0; i < ORD; ++i) {
        if (i < nx) {
          X[q][i] = row(s_in + i * blk, b, K)[k];
          if (tangent) D[q][i] = row(ds_in + i * blk, b, K)[k];
        }
        if (i >= 1 && i < so && in_blocks > 1) {
          F[q][i] = row(s_in + (so + i - 1) * blk, b, K)[k];
          if (tangent) GJ[q][i] = row(ds_in + (so + i - 1) * blk, b, K)[k];
        }
      }
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
  // nu k^2 per mode and 1 / (a_0 + nu k^2), recomputed only when a_0 changes (the step order, or
  // the step size of a schedule)
  double nk2[Q], inv_m[Q];
  for (int q = 0; q < Q; ++q) {
    const double kk = kwav(P, tid + q * G);
    nk2[q] = P.nu * kk * kk;
    inv_m[q] = 0.0;
  }
  double a0_prev = 0.0;
  for (int j = 1; j <= n_steps; ++j) {
    const int n = n_first + j;
    Coef c = step_coef(P, n);
    if (c.a[0] != a0_prev) {
      for (int q = 0; q < Q; ++q) inv_m[q] = 1.0 / (c.a[0] + nk2[q]);
      a0_prev = c.a[0];
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
      if (traj) row(traj + (size_t)j * blk, b, K)[k] = xn;
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
    if (j < n_steps && P.nonlinear) {
      if (tangent) eval_F_and_jvp(P, s, S2, O2, true);
      else eval_F(P, s);
      for (int q = 0; q < Q; ++q) {
        int k = tid + q * G;
        if (k < K) { F[q][0] = s.O[k]; if (tangent) GJ[q][0] = O2[k]; }
      }
    }
  }
  for (int q = 0; q < Q; ++q) {
    int k = tid + q * G;
    if (k >= K) continue;
    if (x_out) row(x_out, b, K)[k] = tangent ? D[q][0] : X[q][0];
    if (s_out) {
#pragma unroll
      for (int i = 0; i < ORD; ++i) {
        if (i < so) row(s_out + i * blk, b, K)[k] = tangent ? D[q][i] : X[q][i];
        if (i >= 1 && i < so) row(s_out + (so + i - 1) * blk, b, K)[k] = tangent ? GJ[q][i] : F[q][i];
      }
    }
  }
}

// Adjoint sweep (eq. IMEX_adjoint) over indices n = n_hi down to n_lo of a horizon of n_steps steps.
// traj holds X_{n_lo}..X_{n_hi} (X_n at traj + (n - n_lo) * state).  At n = n_steps the cotangent is
// seeded with y_final (NULL: zero) and no vector-Jacobian product is formed.  The adjoint variables
// Y_{n+1}, ..., Y_{n+s} (s = P.order) are carried between launches as blocks of [B][K] complex:
// carry_in (nullable = zero) holds Y_{n_hi+1}, ..., Y_{n_hi+s}; out receives Y_{n_lo}, ..., Y_{n_lo+s-1}
// (out_blocks = s) or, when n_lo = 0, dJ/dX_0 in its first block (the right-hand side at n = 0, with no
// solve) followed by Y_1, ..., Y_{s-1} when out_blocks = s.  Cotangents injected at X_n: seeds
// (indexed by seed_at[n], nullable) and src (nullable, at n = n_hi).
template <int Q, int ORD>
__global__ void __launch_bounds__(64) adjoint_kernel(BurgersParams P, int n_steps, int n_hi, int n_lo,
                                                     const double* __restrict__ traj, const double* __restrict__ y_final,
                                                     const double* __restrict__ carry_in, double* __restrict__ out,
                                                     int out_blocks, const int* __restrict__ seed_at,
                                                     const double* __restrict__ seeds, const double* __restrict__ src) {
  Smem s = carve(P);
  extern __shared__ double2 sm[];
  double2* S2 = sm + 4 * P.L + 2 * P.K;
  const int b = blockIdx.x, K = P.K, G = blockDim.x, tid = threadIdx.x;
  const int nb = gridDim.x;
  const size_t stride = (size_t)nb * 2 * K;
  const int so = P.order;
  double2 Y[Q][ORD];  // Y_{n+1}, ..., Y_{n+ORD}
  const double2 z = make_double2(0.0, 0.0);
  // nu k^2 per mode and 1 / (a_0 + nu k^2) of the current step, recomputed when a_0 changes
  double nk2[Q], inv_m[Q];
  for (int q = 0; q < Q; ++q) {
    const double kk = kwav(P, tid + q * G);
    nk2[q] = P.nu * kk * kk;
    inv_m[q] = 0.0;
  }
  double a0_prev = 0.0;
  for (int q = 0; q < Q; ++q) {
    const int k = tid + q * G;
#pragma unroll
    for (int i = 0; i < ORD; ++i) Y[q][i] = (carry_in && i < so && k < K) ? row(carry_in + i * stride, b, K)[k] : z;
  }
  for (int n = n_hi; n >= n_lo; --n) {
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
      const double2* xn = row(traj + (size_t)(n - n_lo) * stride, b, K);
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
    if (src && n == n_hi) {
      for (int q = 0; q < Q; ++q) {
        int k = tid + q * G;
        if (k < K) lam[q] = cadd(lam[q], row(src, b, K)[k]);
      }
    }
    if (n == 0) {
      for (int q = 0; q < Q; ++q) {
        int k = tid + q * G;
        if (k >= K) continue;
        row(out, b, K)[k] = lam[q];
#pragma unroll
        for (int i = 1; i < ORD; ++i)
          if (i < so && i < out_blocks) row(out + i * stride, b, K)[k] = Y[q][i - 1];
      }
      return;
    }
    {
      const Coef c = step_coef(P, n);
      if (c.a[0] != a0_prev) {
        for (int q = 0; q < Q; ++q) inv_m[q] = 1.0 / (c.a[0] + nk2[q]);
        a0_prev = c.a[0];
      }
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
  for (int q = 0; q < Q; ++q) {
    int k = tid + q * G;
    if (k >= K) continue;
#pragma unroll
    for (int i = 0; i < ORD; ++i)
      if (i < so && i < out_blocks) row(out + i * stride, b, K)[k] = Y[q][i];
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

  // ---- step-size schedule (variable-step SBDF1 / SBDF2) ---------------------------------------
  DevBuf wsched;
  spadj_status set_schedule(Problem* p, int n, const double* dts) {
    if (n == 0) {
      P.ws = nullptr;
      P.ws_len = 0;
      return SPADJ_OK;
    }
    if (P.order > 2) return p->fail(SPADJ_ERR_UNSUPPORTED, "burgers: step-size schedules need SBDF1 or SBDF2");
    for (int i = 0; i < n; ++i)
      if (!(dts[i] > 0.0) || !std::isfinite(dts[i])) return p->fail(SPADJ_ERR_INVALID, "set_dt_schedule: step sizes must be > 0");
    // step n (1-based) spans h = dts[n-1]; from the second step on, SBDF2 with w = h / dts[n-2]
    std::vector<double> w((size_t)n * 5, 0.0);
    for (int k = 1; k <= n; ++k) {
      const double h = dts[k - 1];
      double* r = &w[(size_t)(k - 1) * 5];
      if (k == 1 || P.order == 1) {
        r[0] = 1.0 / h; r[1] = -1.0 / h; r[3] = 1.0;
      } else {
        const double om = h / dts[k - 2];
        r[0] = (1.0 + 2.0 * om) / ((1.0 + om) * h);
        r[1] = -(1.0 + om) / h;
        r[2] = om * om / ((1.0 + om) * h);
        r[3] = 1.0 + om;
        r[4] = -om;
      }
    }
    SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));  // no kernel may still read the old table
    SPADJ_CUDA_TRY(p, wsched.ensure(sizeof(double) * w.size()));
    SPADJ_CUDA_TRY(p, cudaMemcpy(wsched.ptr, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice));
    P.ws = wsched.as<double>();
    P.ws_len = n;
    return SPADJ_OK;
  }
  spadj_status check_horizon(Problem* p, int n_steps) {
    if (P.ws && n_steps > P.ws_len) return p->fail(SPADJ_ERR_INVALID, "burgers: the step-size schedule is shorter than the sweep");
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

  // launches of the segment kernels (forward / tangent segment; adjoint over n_hi..n_lo)
  spadj_status launch_traj(Problem* p, int n_first, int n_steps, const double* s_in, int in_blocks, const double* ds_in,
                           double* x_out, double* s_out, double* trj, int tangent) {
    cudaEvent_t t = p->tic();
    spadj_status s = dispatchQ(p, [&](auto q, auto o) {
      trajectory_kernel<decltype(q)::value, decltype(o)::value><<<B, G, smem, p->stream>>>(
          P, n_first, n_steps, s_in, in_blocks, ds_in, x_out, s_out, trj, tangent);
    });
    p->toc(t, KC_FUSED, (double)B * n_steps * ((tangent ? 3 : 2) * fft_flops() + P.M + 10.0 * P.K));
    return s;
  }
  spadj_status launch_adj(Problem* p, int n_steps, int n_hi, int n_lo, const double* trj, const double* y_final,
                          const double* carry_in, double* out, int out_blocks, const int* seed_at, const double* seeds,
                          const double* src) {
    cudaEvent_t t = p->tic();
    spadj_status s = dispatchQ(p, [&](auto q, auto o) {
      adjoint_kernel<decltype(q)::value, decltype(o)::value><<<B, G, smem, p->stream>>>(
          P, n_steps, n_hi, n_lo, trj, y_final, carry_in, out, out_blocks, seed_at, seeds, src);
    });
    p->toc(t, KC_FUSED, (double)B * (n_hi - n_lo + 1) * (3 * fft_flops() + 2.0 * P.M + 12.0 * P.K));
    return s;
  }

  spadj_status forward(Problem* p, int n_steps, const double* x0, double* x_out, double* trj) override {
    if (n_steps < 0) return p->fail(SPADJ_ERR_INVALID, "forward: n_steps < 0");
    if (spadj_status h = check_horizon(p, n_steps)) return h;
    return launch_traj(p, 0, n_steps, x0, 1, nullptr, x_out, nullptr, trj, 0);
  }

  spadj_status tangent(Problem* p, int n_steps, const double* x0, const double* dx0, double* dx_out) override {
    if (n_steps < 0) return p->fail(SPADJ_ERR_INVALID, "tangent: n_steps < 0");
    if (spadj_status h = check_horizon(p, n_steps)) return h;
    return launch_traj(p, 0, n_steps, x0, 1, dx0, dx_out, nullptr, nullptr, 1);
  }

  // ---- one step at a time ----------------------------------------------------------------------
  // restart state: 2s - 1 blocks [X_n..X_{n-s+1}, F(X_{n-1})..F(X_{n-s+1})]; adjoint state: s blocks
  // [Y_n..Y_{n+s-1}] (the adjoint variables of eq. IMEX_adjoint), s = the scheme's order
  int step_blocks(int which) const override { return which == 0 ? 2 * P.order - 1 : P.order; }

  spadj_status step_forward(Problem* p, int n, const double* s_n, double* s_np1) override {
    if (n < 0) return p->fail(SPADJ_ERR_INVALID, "step: n < 0");
    if (spadj_status h = check_horizon(p, n + 1)) return h;
    return launch_traj(p, n, 1, s_n, 2 * P.order - 1, nullptr, nullptr, s_np1, nullptr, 0);
  }

  spadj_status step_tangent(Problem* p, int n, const double* s_n, const double* ds_n, double* ds_np1) override {
    if (n < 0) return p->fail(SPADJ_ERR_INVALID, "step: n < 0");
    if (spadj_status h = check_horizon(p, n + 1)) return h;
    return launch_traj(p, n, 1, s_n, 2 * P.order - 1, ds_n, nullptr, ds_np1, nullptr, 1);
  }

  spadj_status step_adjoint(Problem* p, int n, const double* x_n, const double* y_np1, const double* src, double* y_n,
                            double* gp_accum) override {
    if (gp_accum) return p->fail(SPADJ_ERR_INVALID, "burgers: the problem has no parameters (gp_accum must be NULL)");
    if (n < 0) return p->fail(SPADJ_ERR_INVALID, "step: n < 0");
    if (spadj_status h = check_horizon(p, n)) return h;
    // y_np1 = NULL: the seed step (no later adjoint variables); otherwise every later step exists and
    // the adjoint variables past the horizon are the caller's zeros
    const int horizon = y_np1 ? (1 << 29) : n;
    return launch_adj(p, horizon, n, n, x_n, nullptr, y_np1, y_n, P.order, nullptr, nullptr, src);
  }

  // ---- reverse sweeps ------------------------------------------------------------------------------
  DevBuf rs, ys, slots, seedmap;  // restart-state ping-pong, adjoint-state ping-pong, checkpoint slots
  HostBuf hslots;
  int last_recompute = 0;

  // Reverse sweep of n_steps steps.  y_final (nullable) seeds dJ/dX_N; seed_at[n] (nullable, host)
  // indexes `seeds` for cotangents injected at X_n.  ckpt_slots <= 0 or > n_steps: the whole trajectory
  // is stored and reversed in one launch; otherwise the binomial schedule (two-level with host slots,
  // spadj_set_option 9) over device slots that hold full restart states, each forward segment and each
  // adjoint step one launch over all members, the adjoint state carried between launches.
  spadj_status reverse(Problem* p, const double* x0, int n_steps, int ckpt_slots, const double* y_final_dev,
                       const std::vector<int>* seed_at, const double* seeds, double* grad, double* J_dev,
                       double* seed_buf) {
    if (spadj_status h = check_horizon(p, n_steps)) return h;
    const size_t sl = state_len(0);
    const int* sm_dev = nullptr;
    if (seed_at) {
      SPADJ_CUDA_TRY(p, seedmap.ensure(sizeof(int) * (size_t)(n_steps + 1)));
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(seedmap.ptr, seed_at->data(), sizeof(int) * (n_steps + 1),
                                        cudaMemcpyHostToDevice, p->stream));
      sm_dev = seedmap.as<int>();
    }
    spadj_status st;
    const int S = (ckpt_slots <= 0 || ckpt_slots > n_steps) ? n_steps + 1 : ckpt_slots;
    if (S == n_steps + 1) {  // store-all: one forward launch, one adjoint launch
      SPADJ_CUDA_TRY(p, traj.ensure(sizeof(double) * sl * (size_t)(n_steps + 1)));
      double* T = traj.as<double>();
      double* xN = T + (size_t)n_steps * sl;
      if ((st = forward(p, n_steps, x0, xN, T)) != SPADJ_OK) return st;
      const double* yf = y_final_dev;
      if (J_dev) {
        if ((st = this->objective(p, SPADJ_OBJ_ENERGY, nullptr, xN, J_dev, seed_buf)) != SPADJ_OK) return st;
        yf = seed_buf;
      }
      st = launch_adj(p, n_steps, n_steps, 0, T, yf, nullptr, grad, 1, sm_dev, seeds, nullptr);
      if (st == SPADJ_OK && seed_at) SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));  // pageable staging
      return st;
    }
    const int so = P.order, rb = 2 * so - 1;
    const size_t rbytes = sizeof(double) * sl * rb, ybytes = sizeof(double) * sl * so;
    SPADJ_CUDA_TRY(p, rs.ensure(2 * rbytes));
    SPADJ_CUDA_TRY(p, ys.ensure(2 * ybytes));
    SPADJ_CUDA_TRY(p, slots.ensure(rbytes * (size_t)S));
    CkptPlanner planner;
    const int H = std::min(p->host_slots, n_steps);
    std::vector<CkptOp> ops = H > 0 ? planner.plan2(n_steps, S, H) : planner.plan(n_steps, S);
    if (H > 0) SPADJ_CUDA_TRY(p, hslots.ensure(rbytes * (size_t)H));
    auto slot_ptr = [&](int k) {
      return k < S ? slots.as<char>() + (size_t)k * rbytes : hslots.as<char>() + (size_t)(k - S) * rbytes;
    };
    double* R[2] = {rs.as<double>(), rs.as<double>() + sl * rb};
    double* Yc[2] = {ys.as<double>(), ys.as<double>() + sl * so};
    int ri = 0, yi = 0, recompute = 0, cur_step = 0;
    bool have_seed = false;
    // the restart state of X_0: X_0 and zero history
    SPADJ_CUDA_TRY(p, cudaMemsetAsync(R[ri], 0, rbytes, p->stream));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(R[ri], x0, sizeof(double) * sl, cudaMemcpyDeviceToDevice, p->stream));
    for (const CkptOp& op : ops) {
      switch (op.type) {
        case CK_STORE:
          SPADJ_CUDA_TRY(p, cudaMemcpyAsync(slot_ptr(op.slot), R[ri], rbytes,
                                            op.slot < S ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream));
          break;
        case CK_RESTORE:
          if (cur_step != op.a) {
            SPADJ_CUDA_TRY(p, cudaMemcpyAsync(R[ri], slot_ptr(op.slot), rbytes,
                                              op.slot < S ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                              p->stream));
            cur_step = op.a;
          }
          break;
        case CK_ADVANCE:
          if ((st = launch_traj(p, op.a, op.b - op.a, R[ri], rb, nullptr, nullptr, R[1 - ri], nullptr, 0)) != SPADJ_OK)
            return st;
          ri = 1 - ri;
          recompute += op.b - op.a;
          cur_step = op.b;
          break;
        case CK_OBJECTIVE: {
          const double* yf = y_final_dev;
          if (J_dev) {
            if ((st = this->objective(p, SPADJ_OBJ_ENERGY, nullptr, R[ri], J_dev, seed_buf)) != SPADJ_OK) return st;
            yf = seed_buf;
          }
          if ((st = launch_adj(p, n_steps, n_steps, n_steps, R[ri], yf, nullptr, Yc[yi], so, sm_dev, seeds, nullptr)) !=
              SPADJ_OK)
            return st;
          have_seed = true;
          break;
        }
        case CK_ADJOINT: {
          if (!have_seed) return p->fail(SPADJ_ERR_INVALID, "gradient: schedule reached an adjoint step before the objective");
          double* out = op.a == 0 ? grad : Yc[1 - yi];
          if ((st = launch_adj(p, n_steps, op.a, op.a, R[ri], nullptr, Yc[yi], out, op.a == 0 ? 1 : so, sm_dev, seeds,
                               nullptr)) != SPADJ_OK)
            return st;
          yi = 1 - yi;
          break;
        }
        default:
          break;
      }
    }
    last_recompute = recompute;
    if (seed_at || H > 0) SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));  // pageable staging, host slots
    return SPADJ_OK;
  }

  spadj_status vjp(Problem* p, const double* x0, int n_steps, int ckpt_slots, const std::vector<int>& seed_at,
                   const double* seeds, double* grad) override {
    if (n_steps < 1) return p->fail(SPADJ_ERR_INVALID, "vjp: n_steps < 1");
    return reverse(p, x0, n_steps, ckpt_slots, nullptr, &seed_at, seeds, grad, nullptr, nullptr);
  }

  spadj_status adjoint(Problem* p, int n_steps, const double* trj, const double* y_final, double* grad,
                       double* grad_p) override {
    if (n_steps < 1) return p->fail(SPADJ_ERR_INVALID, "adjoint: n_steps < 1");
    if (grad_p) return p->fail(SPADJ_ERR_INVALID, "burgers: the problem has no parameters (grad_p must be NULL)");
    if (spadj_status h = check_horizon(p, n_steps)) return h;
    return launch_adj(p, n_steps, n_steps, 0, trj, y_final, nullptr, grad, 1, nullptr, nullptr, nullptr);
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
    (void)obj_data;
    if (grad_p) return p->fail(SPADJ_ERR_INVALID, "burgers: the problem has no parameters (grad_p must be NULL)");
    if (objective != SPADJ_OBJ_ENERGY) return p->fail(SPADJ_ERR_UNSUPPORTED, "burgers: objective must be ENERGY");
    if (n_steps < 1) return p->fail(SPADJ_ERR_INVALID, "gradient: n_steps < 1");
    const size_t sl = state_len(0);
    SPADJ_CUDA_TRY(p, seed.ensure(sizeof(double) * sl));
    SPADJ_CUDA_TRY(p, Jd.ensure(sizeof(double) * B));
    spadj_status st = reverse(p, x0, n_steps, ckpt_slots, nullptr, nullptr, nullptr, grad, Jd.as<double>(),
                              seed.as<double>());
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
    wsched.release();
    seedmap.release();
    rs.release();
    ys.release();
    slots.release();
    hslots.release();
    traj.release();
    seed.release();
    Jd.release();
  }
};

}  // namespace

spadj_status burgers_set_dt_schedule(EqImpl* impl, Problem* p, int n, const double* dts) {
  Burgers* b = dynamic_cast<Burgers*>(impl);
  if (!b) return p->fail(SPADJ_ERR_UNSUPPORTED, "set_dt_schedule: not a Burgers problem");
  return b->set_schedule(p, n, dts);
}

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
