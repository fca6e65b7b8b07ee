// Host-side construction of the Rayleigh-Benard pencil operators and of the per-pencil
// prognostic solution operators (run once per problem, off the per-step path).
//
// Discretisation (Sparse spectral methods section; Supplementary A.4 IVP form): per
// x-wavenumber k the unknowns are the Chebyshev-T coefficients of u, w, theta, p
// (N each) and seven tau variables; momentum and temperature rows are projected on the
// ultraspherical C^(2) basis, continuity on C^(1); boundary rows evaluate T_n(+-1); the
// kx = 0 pencil carries the pressure gauge int p dz = 0 and its tau.  The implicit
// matrix of one RK222 stage is A = M + dt*gamma*L (both stages share it).
//
// Every right-hand side the timestepper builds has the form [S1S0 v_u; S1S0 v_w;
// S1S0 v_t; 0...] with v in T space, and only the prognostic block of the solution is
// used afterwards, so the stage solve is the linear map
//     Phi = [A^-1]_{prognostic cols of x, prognostic rows of R} * blockdiag(S1S0)
// (3N x 3N per pencil).  With the substitution u = i*u~ (u-momentum and u-boundary rows
// scaled by -i, u and tau_u columns by i) every pencil matrix is real, so Phi = Dc Phi' Dr
// with Phi' real; Phi' is computed here by LU with partial pivoting of the real pencil
// matrix (the paper reuses one factorisation per timestep size, Methods "Linear system
// solves") and applied on the GPU as a dense matvec.
#include <cmath>
#include <thread>
#include <vector>

#include "rb_setup.h"

namespace spadj {
namespace rbhost {

namespace {
using Mat = std::vector<double>;  // row-major
}  // namespace

// d/dxi T_n = n C1_{n-1}
std::vector<double> op_D0(int N, double s) {
  Mat m(N * N, 0.0);
  for (int n = 1; n < N; ++n) m[(n - 1) * N + n] = n * s;
  return m;
}
// d/dxi C1_n = 2 C2_{n-1}
std::vector<double> op_D1(int N, double s) {
  Mat m(N * N, 0.0);
  for (int n = 1; n < N; ++n) m[(n - 1) * N + n] = 2.0 * s;
  return m;
}
// T -> C1 conversion
std::vector<double> op_S0(int N) {
  Mat m(N * N, 0.0);
  m[0] = 1.0;
  if (N > 1) m[1 * N + 1] = 0.5;
  for (int n = 2; n < N; ++n) {
    m[n * N + n] = 0.5;
    m[(n - 2) * N + n] = -0.5;
  }
  return m;
}
// C1 -> C2 conversion
std::vector<double> op_S1(int N) {
  Mat m(N * N, 0.0);
  for (int n = 0; n < N; ++n) {
    m[n * N + n] = 1.0 / (n + 1);
    if (n >= 2) m[(n - 2) * N + n] = -1.0 / (n + 1);
  }
  return m;
}
std::vector<double> matmul(const std::vector<double>& a, const std::vector<double>& b, int N) {
  Mat c(N * N, 0.0);
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < N; ++k) {
      double v = a[i * N + k];
      if (v == 0.0) continue;
      for (int j = 0; j < N; ++j) c[i * N + j] += v * b[k * N + j];
    }
  return c;
}

namespace {

// In-place LU with partial pivoting of an n x n row-major matrix; returns false if singular.
bool lu_factor(std::vector<double>& a, std::vector<int>& piv, int n) {
  piv.resize(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(a[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = std::fabs(a[(size_t)i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    if (best == 0.0) return false;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)p * n + j]);
    const double inv = 1.0 / a[(size_t)k * n + k];
    for (int i = k + 1; i < n; ++i) {
      double l = a[(size_t)i * n + k] * inv;
      a[(size_t)i * n + k] = l;
      if (l == 0.0) continue;
      double* ri = &a[(size_t)i * n];
      const double* rk = &a[(size_t)k * n];
      for (int j = k + 1; j < n; ++j) ri[j] -= l * rk[j];
    }
  }
  return true;
}

// Solve A x = b (b overwritten) with the factors of lu_factor.
void lu_solve(const std::vector<double>& a, const std::vector<int>& piv, int n, double* b) {
  for (int k = 0; k < n; ++k) {
    if (piv[k] != k) std::swap(b[k], b[piv[k]]);
  }
  for (int i = 1; i < n; ++i) {
    double s = b[i];
    const double* ri = &a[(size_t)i * n];
    for (int j = 0; j < i; ++j) s -= ri[j] * b[j];
    b[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    const double* ri = &a[(size_t)i * n];
    for (int j = i + 1; j < n; ++j) s -= ri[j] * b[j];
    b[i] = s / ri[i];
  }
}

}  // namespace

Operators build_operators(int N, int Mz, double zs) {
  Operators o;
  o.N = N;
  o.Mz = Mz;
  Mat S0 = op_S0(N), S1 = op_S1(N), D0 = op_D0(N, zs), D1 = op_D1(N, zs);
  o.SS = matmul(S1, S0, N);
  o.DD = matmul(D1, D0, N);
  o.SD = matmul(S1, D0, N);
  o.S0 = S0;
  o.D0 = D0;
  o.lift_row = N - 2;           // d/dz of the last C^(1) mode lands on C^(2) mode N-2
  o.lift_val = D1[(N - 2) * N + (N - 1)];
  // derivative in the T basis, Dz = S0^-1 D0 (back substitution on upper-triangular S0)
  o.Dz.assign(N * N, 0.0);
  for (int col = 0; col < N; ++col) {
    for (int i = N - 1; i >= 0; --i) {
      double s = D0[i * N + col];
      for (int j = i + 1; j < N; ++j) s -= S0[i * N + j] * o.Dz[j * N + col];
      o.Dz[i * N + col] = s / S0[i * N + i];
    }
  }
  // Gauss-Chebyshev grid xi_j = -cos(pi (j + 1/2) / Mz) and transform matrices
  o.Cz.assign((size_t)Mz * N, 0.0);
  o.Gz.assign((size_t)N * Mz, 0.0);
  for (int j = 0; j < Mz; ++j) {
    const double theta = M_PI - M_PI * (j + 0.5) / Mz;  // arccos(xi_j)
    for (int n = 0; n < N; ++n) {
      const double t = std::cos(n * theta);
      o.Cz[(size_t)j * N + n] = t;
      o.Gz[(size_t)n * Mz + j] = (n == 0 ? 1.0 : 2.0) * t / Mz;
    }
  }
  // C'z = Cz Dz: values of dz T_n on the grid
  o.Cdz.assign((size_t)Mz * N, 0.0);
  for (int j = 0; j < Mz; ++j)
    for (int n = 0; n < N; ++n) {
      double s = 0.0;
      for (int k = 0; k < N; ++k) s += o.Cz[(size_t)j * N + k] * o.Dz[k * N + n];
      o.Cdz[(size_t)j * N + n] = s;
    }
  // int T_m T_n dz over the interval = (1/zs) int_{-1}^{1} T_m T_n dxi = (I_{m+n} + I_{|m-n|}) / (2 zs)
  auto I = [](int k) { return (k % 2 == 0) ? 2.0 / (1.0 - (double)k * k) : 0.0; };
  o.G.assign(N * N, 0.0);
  for (int m = 0; m < N; ++m)
    for (int n = 0; n < N; ++n) o.G[m * N + n] = (0.5 / zs) * (I(m + n) + I(std::abs(m - n)));
  return o;
}

// Real pencil matrix A' = Dr (M + b L) Dc for wavenumber k (u-rows/u-BC rows times -i,
// u/tau_u columns times i).  Ordering as documented in rb_setup.h.
static void assemble_real_pencil(const Operators& o, double k, bool mean, double nu, double kappa, double b,
                                 std::vector<double>& A) {
  const int N = o.N, nv = 4 * N + 7;
  A.assign((size_t)nv * nv, 0.0);
  auto at = [&](int r, int c) -> double& { return A[(size_t)r * nv + c]; };
  const int U = 0, W = N, T = 2 * N, P = 3 * N;
  const int tu1 = 4 * N, tu2 = 4 * N + 1, tw1 = 4 * N + 2, tw2 = 4 * N + 3, tt1 = 4 * N + 4, tt2 = 4 * N + 5,
            tp = 4 * N + 6;
  const double k2 = k * k;
  for (int r = 0; r < N; ++r)
    for (int c = 0; c < N; ++c) {
      const double ss = o.SS[r * N + c], dd = o.DD[r * N + c];
      // M + b L with L_q = -D_q (DD - k^2 SS); u block: (-i)(.)(i) = identity scaling
      at(U + r, U + c) = ss + b * (-nu) * (dd - k2 * ss);
      at(W + r, W + c) = ss + b * (-nu) * (dd - k2 * ss);
      at(T + r, T + c) = ss + b * (-kappa) * (dd - k2 * ss);
      // u-eq pressure: b * i k SS, row times -i -> b k SS
      at(U + r, P + c) = b * k * ss;
      // w-eq: b (SD p - SS theta)
      at(W + r, P + c) = b * o.SD[r * N + c];
      at(W + r, T + c) = -b * ss;
      // theta-eq: -b SS w
      at(T + r, W + c) = -b * ss;
      // continuity (C^(1) rows): b (i k S0 u + D0 w), u column times i -> -b k S0
      at(P + r, U + c) = -b * k * o.S0[r * N + c];
      at(P + r, W + c) = b * o.D0[r * N + c];
    }
  // tau terms (part of L, scaled by b); u-eq rows times -i and tau_u columns times i cancel
  // -D_q d/dz(lift(tau_q1)): the lift column enters the q-row with -D_q * lift_val
  at(U + o.lift_row, tu1) = -b * nu * o.lift_val;
  at(U + N - 1, tu2) = b;
  at(W + o.lift_row, tw1) = -b * nu * o.lift_val;
  at(W + N - 1, tw2) = b;
  at(T + o.lift_row, tt1) = -b * kappa * o.lift_val;
  at(T + N - 1, tt2) = b;
  at(P + N - 1, tw1) = b;
  // boundary rows (in L): u rows times -i, u columns times i -> real
  const int r0 = 4 * N;
  for (int n = 0; n < N; ++n) {
    const double bot = (n % 2 == 0) ? 1.0 : -1.0;
    at(r0 + 0, U + n) = b * bot;
    at(r0 + 1, U + n) = b;
    at(r0 + 2, W + n) = b * bot;
    at(r0 + 3, W + n) = b;
    at(r0 + 4, T + n) = b * bot;
    at(r0 + 5, T + n) = b;
  }
  if (mean) {
    at(P + 0, tp) = b;
    for (int n = 0; n < N; n += 2) at(r0 + 6, P + n) = b * 2.0 / (1.0 - (double)n * n);
  } else {
    at(r0 + 6, tp) = b;
  }
}

bool build_phi(const Operators& o, int Kx, double Lx, double nu, double kappa, double b, std::vector<double>& phi,
               std::string* err) {
  const int N = o.N, nv = 4 * N + 7, np = 3 * N;
  phi.assign((size_t)Kx * np * np, 0.0);
  std::vector<int> bad(Kx, 0);
  auto work = [&](int m0, int m1) {
    std::vector<double> A, rhs(nv);
    std::vector<int> piv;
    for (int m = m0; m < m1; ++m) {
      const double k = 2.0 * M_PI * m / Lx;
      assemble_real_pencil(o, k, m == 0, nu, kappa, b, A);
      if (!lu_factor(A, piv, nv)) {
        bad[m] = 1;
        continue;
      }
      double* out = &phi[(size_t)m * np * np];
      // column c of Phi': solve with RHS = SS column placed in the rows of its field
      for (int f = 0; f < 3; ++f)
        for (int c = 0; c < N; ++c) {
          std::fill(rhs.begin(), rhs.end(), 0.0);
          for (int r = 0; r < N; ++r) rhs[f * N + r] = o.SS[r * N + c];
          lu_solve(A, piv, nv, rhs.data());
          for (int r = 0; r < np; ++r) out[(size_t)r * np + f * N + c] = rhs[r];
        }
    }
  };
  unsigned nt = std::thread::hardware_concurrency();
  if (nt == 0) nt = 1;
  if (nt > 32) nt = 32;
  if ((int)nt > Kx) nt = Kx;
  std::vector<std::thread> th;
  const int chunk = (Kx + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    int m0 = t * chunk, m1 = std::min(Kx, m0 + chunk);
    if (m0 < m1) th.emplace_back(work, m0, m1);
  }
  for (auto& t : th) t.join();
  for (int m = 0; m < Kx; ++m)
    if (bad[m]) {
      if (err) *err = "rb: singular pencil matrix at kx index " + std::to_string(m);
      return false;
    }
  return true;
}

}  // namespace rbhost
}  // namespace spadj
