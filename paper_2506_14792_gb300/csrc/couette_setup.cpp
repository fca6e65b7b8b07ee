// Host-side construction of the plane-Couette per-pencil solution operators (once per
// problem and timestep scheme, off the per-step path).
//
// Perturbation equations about U(z) = z on z in [-1, 1] (Supplementary A.4 IVP form):
//   dt u - nu lap u + U dx u + w U' e_x + grad p = F,   div u = 0,   u = 0 at z = +-1.
// Per wavenumber pair (kx, ky) the Chebyshev-T coefficients of u, v, w, p and seven tau
// variables are the unknowns (Sparse spectral methods section): momentum rows on C^(2),
// continuity on C^(1), first-order tau lifts (tau_q1 through d/dz of the last C^(1) mode,
// tau_q2 on the last C^(2) mode, tau_w1 also in the last continuity row), boundary rows
// T_n(+-1), and the gauge int p dz = 0 with tau_p on the mean pencil.  The advection
// U dx = i kx z is the exact product z T_n (degree N) converted with S1 S0 and truncated.
//
// A multistep right-hand side is [S1S0 v_u; S1S0 v_v; S1S0 v_w; 0...] with v in T space
// (b_i = 0 for i >= 1), and only the prognostic block of the solution is used, so the step
// solve is the linear map Phi (3N x 3N per pencil).  The pencil matrix is complex (the
// advection term is imaginary), so Phi is complex; it is computed here by LU with partial
// pivoting (one factorisation per pencil and scheme, reused every step: Methods "Linear
// system solves") and applied on the GPU as a dense matvec.  The banded form (build_band)
// keeps the factors instead: the pencil matrix, recombined so that its boundary rows become
// local and ordered by Chebyshev mode, is narrowly banded (Sparse spectral methods section), and
// the GPU runs its forward and back sweeps.
#include "couette_setup.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <thread>
#include <tuple>

namespace spadj {
namespace couhost {

using cd = std::complex<double>;

namespace {
// y -= l x over n complex entries, written on the interleaved (re, im) doubles so that the
// compiler vectorises it (std::complex products carry a NaN-recovery branch that blocks it)
inline void caxpy_sub(cd* y, const cd* x, cd l, int n) {
  double* __restrict yd = reinterpret_cast<double*>(y);
  const double* __restrict xd = reinterpret_cast<const double*>(x);
  const double lr = l.real(), li = l.imag();
  for (int c = 0; c < n; ++c) {
    const double xr = xd[2 * c], xi = xd[2 * c + 1];
    yd[2 * c] -= lr * xr - li * xi;
    yd[2 * c + 1] -= lr * xi + li * xr;
  }
}
}  // namespace

bool lu_factor(std::vector<cd>& a, std::vector<int>& piv, int n) {
  piv.resize(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::abs(a[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      const double v = std::abs(a[(size_t)i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    if (best == 0.0) return false;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)p * n + j]);
    const cd inv = 1.0 / a[(size_t)k * n + k];
    const cd* rk = &a[(size_t)k * n];
    for (int i = k + 1; i < n; ++i) {
      const cd l = a[(size_t)i * n + k] * inv;
      a[(size_t)i * n + k] = l;
      if (l == 0.0) continue;
      caxpy_sub(&a[(size_t)i * n + k + 1], rk + k + 1, l, n - k - 1);
    }
  }
  return true;
}

// Right-hand sides are swept in panels of kPanel columns, so that the rows of a panel stay in
// cache through a whole substitution (the arithmetic of every entry is unchanged).
constexpr int kPanel = 32;

// Solve A X = B for nr right-hand sides held row-major in B (n x nr), overwritten.
void lu_solve_multi(const std::vector<cd>& a, const std::vector<int>& piv, int n, std::vector<cd>& B, int nr) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k)
      for (int c = 0; c < nr; ++c) std::swap(B[(size_t)k * nr + c], B[(size_t)piv[k] * nr + c]);
  for (int c0 = 0; c0 < nr; c0 += kPanel) {
    const int w = std::min(kPanel, nr - c0);
    for (int i = 1; i < n; ++i) {
      cd* bi = &B[(size_t)i * nr + c0];
      for (int j = 0; j < i; ++j) {
        const cd l = a[(size_t)i * n + j];
        if (l == 0.0) continue;
        caxpy_sub(bi, &B[(size_t)j * nr + c0], l, w);
      }
    }
    for (int i = n - 1; i >= 0; --i) {
      cd* bi = &B[(size_t)i * nr + c0];
      for (int j = i + 1; j < n; ++j) {
        const cd u = a[(size_t)i * n + j];
        if (u == 0.0) continue;
        caxpy_sub(bi, &B[(size_t)j * nr + c0], u, w);
      }
      const cd inv = 1.0 / a[(size_t)i * n + i];
      for (int c = 0; c < w; ++c) bi[c] *= inv;
    }
  }
}

// Solve A^H X = B with the factors of A from lu_factor (P A = L U, so A^H = U^H L^H P):
// forward substitution with U^H, back substitution with the unit L^H, then the row swaps
// undone in reverse order.
void lu_solve_h_multi(const std::vector<cd>& a, const std::vector<int>& piv, int n, std::vector<cd>& B, int nr) {
  for (int c0 = 0; c0 < nr; c0 += kPanel) {
    const int w = std::min(kPanel, nr - c0);
    for (int i = 0; i < n; ++i) {
      cd* bi = &B[(size_t)i * nr + c0];
      for (int j = 0; j < i; ++j) {
        const cd u = std::conj(a[(size_t)j * n + i]);
        if (u == 0.0) continue;
        caxpy_sub(bi, &B[(size_t)j * nr + c0], u, w);
      }
      const cd inv = 1.0 / std::conj(a[(size_t)i * n + i]);
      for (int c = 0; c < w; ++c) bi[c] *= inv;
    }
    for (int i = n - 2; i >= 0; --i) {
      cd* bi = &B[(size_t)i * nr + c0];
      for (int j = i + 1; j < n; ++j) {
        const cd l = std::conj(a[(size_t)j * n + i]);
        if (l == 0.0) continue;
        caxpy_sub(bi, &B[(size_t)j * nr + c0], l, w);
      }
    }
  }
  for (int k = n - 1; k >= 0; --k)
    if (piv[k] != k)
      for (int c = 0; c < nr; ++c) std::swap(B[(size_t)k * nr + c], B[(size_t)piv[k] * nr + c]);
}

void base_flow(const rbhost::Operators& o, int base, std::vector<double>& Umat, std::vector<double>& UPmat) {
  const int N = o.N;
  // ZS = (S1 S0 on N + 1 modes) * (z T_n in the T basis of degree N), first N rows
  std::vector<double> S0e = rbhost::op_S0(N + 1), S1e = rbhost::op_S1(N + 1);
  std::vector<double> SSe = rbhost::matmul(S1e, S0e, N + 1);
  std::vector<double> ZS((size_t)N * N, 0.0);
  for (int r = 0; r < N; ++r)
    for (int n = 0; n < N; ++n) {
      // z T_0 = T_1; z T_n = (T_{n+1} + T_{n-1}) / 2
      double v = 0.0;
      if (n == 0) {
        v = SSe[(size_t)r * (N + 1) + 1];
      } else {
        v = 0.5 * (SSe[(size_t)r * (N + 1) + n + 1] + SSe[(size_t)r * (N + 1) + n - 1]);
      }
      ZS[(size_t)r * N + n] = v;
    }
  if (base == 0) {  // U = z, U' = 1
    Umat = ZS;
    UPmat = o.SS;
    return;
  }
  // U = 1 - z^2: (1 - z^2) T_n in the T basis of degree N + 1 (z applied twice), converted
  // with S1 S0 on N + 2 modes and truncated; U' = -2 z
  const int E = N + 2;
  std::vector<double> S2 = rbhost::matmul(rbhost::op_S1(E), rbhost::op_S0(E), E);
  Umat.assign((size_t)N * N, 0.0);
  UPmat.assign((size_t)N * N, 0.0);
  std::vector<double> t(E), z1(E), z2(E);
  auto zmul = [&](const std::vector<double>& in, std::vector<double>& out) {
    std::fill(out.begin(), out.end(), 0.0);
    for (int k = 0; k + 1 < E; ++k) {
      if (in[k] == 0.0) continue;
      if (k == 0) {
        out[1] += in[0];
      } else {
        out[k + 1] += 0.5 * in[k];
        out[k - 1] += 0.5 * in[k];
      }
    }
  };
  for (int n = 0; n < N; ++n) {
    std::fill(t.begin(), t.end(), 0.0);
    t[n] = 1.0;
    zmul(t, z1);
    zmul(z1, z2);
    for (int r = 0; r < N; ++r) {
      double u = 0.0;
      for (int k = 0; k < E; ++k) u += S2[(size_t)r * E + k] * (t[k] - z2[k]);
      Umat[(size_t)r * N + n] = u;
      UPmat[(size_t)r * N + n] = -2.0 * ZS[(size_t)r * N + n];
    }
  }
}

// a0 M + L for the pencil (alpha, beta); ordering as documented in couette_setup.h.
void assemble_pencil(const rbhost::Operators& o, const std::vector<double>& ZS, const std::vector<double>& UP,
                     double al, double be, bool mean, double nu, cd a0, std::vector<cd>& A) {
  const int N = o.N, nv = 4 * N + 7;
  A.assign((size_t)nv * nv, cd(0.0, 0.0));
  auto at = [&](int r, int c) -> cd& { return A[(size_t)r * nv + c]; };
  const int U = 0, V = N, W = 2 * N, P = 3 * N;
  const int tu1 = 4 * N, tu2 = tu1 + 1, tv1 = tu1 + 2, tv2 = tu1 + 3, tw1 = tu1 + 4, tw2 = tu1 + 5, tp = tu1 + 6;
  const double k2 = al * al + be * be;
  const cd ia(0.0, al), ib(0.0, be);
  for (int r = 0; r < N; ++r)
    for (int c = 0; c < N; ++c) {
      const double ss = o.SS[r * N + c], dd = o.DD[r * N + c];
      const cd diag = a0 * ss - nu * (dd - k2 * ss) + ia * ZS[r * N + c];
      at(U + r, U + c) = diag;
      at(V + r, V + c) = diag;
      at(W + r, W + c) = diag;
      at(U + r, W + c) = UP[r * N + c];  // w U' e_x
      at(U + r, P + c) = ia * ss;       // dx p
      at(V + r, P + c) = ib * ss;       // dy p
      at(W + r, P + c) = o.SD[r * N + c];  // dz p
      at(P + r, U + c) = ia * o.S0[r * N + c];  // continuity (C^(1) rows)
      at(P + r, V + c) = ib * o.S0[r * N + c];
      at(P + r, W + c) = o.D0[r * N + c];
    }
  // -nu d/dz(lift(tau_q1)) enters row N-2 of the q-equation with -nu * lift_val
  at(U + o.lift_row, tu1) = -nu * o.lift_val;
  at(V + o.lift_row, tv1) = -nu * o.lift_val;
  at(W + o.lift_row, tw1) = -nu * o.lift_val;
  at(U + N - 1, tu2) = 1.0;
  at(V + N - 1, tv2) = 1.0;
  at(W + N - 1, tw2) = 1.0;
  at(P + N - 1, tw1) = 1.0;
  const int r0 = 4 * N;
  for (int n = 0; n < N; ++n) {
    const double bot = (n % 2 == 0) ? 1.0 : -1.0;
    at(r0 + 0, U + n) = bot;
    at(r0 + 1, U + n) = 1.0;
    at(r0 + 2, V + n) = bot;
    at(r0 + 3, V + n) = 1.0;
    at(r0 + 4, W + n) = bot;
    at(r0 + 5, W + n) = 1.0;
  }
  if (mean) {
    at(P + 0, tp) = 1.0;
    for (int n = 0; n < N; n += 2) at(r0 + 6, P + n) = 2.0 / (1.0 - (double)n * n);
  } else {
    at(r0 + 6, tp) = 1.0;
  }
}

bool build_phi(const rbhost::Operators& o, int Kx, int Ny, double Lx, double Ly, double nu, cd a0,
               std::vector<double>& phiF, std::vector<double>& phiA, std::string* err, int base) {
  const int N = o.N, nv = 4 * N + 7, H = 3 * N, Nyh = Ny / 2;
  std::vector<double> ZS, UP;
  base_flow(o, base, ZS, UP);
  const size_t per = (size_t)H * H * 2;
  const int npen = Kx * Nyh;
  phiF.assign((size_t)npen * per, 0.0);
  phiA.assign((size_t)npen * per, 0.0);
  std::vector<int> bad(npen, 0);
  auto work = [&](int p0, int p1) {
    std::vector<cd> A, B;
    std::vector<int> piv;
    for (int pp = p0; pp < p1; ++pp) {
      const int jh = pp / Kx, m = pp % Kx;
      const double al = 2.0 * M_PI / Lx * m, be = 2.0 * M_PI / Ly * jh;
      assemble_pencil(o, ZS, UP, al, be, m == 0 && jh == 0, nu, a0, A);
      if (!lu_factor(A, piv, nv)) {
        bad[pp] = 1;
        continue;
      }
      B.assign((size_t)nv * H, cd(0.0, 0.0));
      for (int f = 0; f < 3; ++f)
        for (int c = 0; c < N; ++c)
          for (int r = 0; r < N; ++r) B[(size_t)(f * N + r) * H + f * N + c] = o.SS[r * N + c];
      lu_solve_multi(A, piv, nv, B, H);
      double* F = &phiF[(size_t)pp * per];
      double* Aa = &phiA[(size_t)pp * per];
      for (int r = 0; r < H; ++r)
        for (int k = 0; k < H; ++k) {
          const cd v = B[(size_t)r * H + k];
          F[2 * ((size_t)k * H + r)] = v.real();
          F[2 * ((size_t)k * H + r) + 1] = v.imag();
          Aa[2 * ((size_t)r * H + k)] = v.real();
          Aa[2 * ((size_t)r * H + k) + 1] = v.imag();
        }
    }
  };
  unsigned nt = std::thread::hardware_concurrency();
  if (nt == 0) nt = 1;
  if (nt > 64) nt = 64;
  if ((int)nt > npen) nt = npen;
  std::vector<std::thread> th;
  const int chunk = (npen + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    const int p0 = t * chunk, p1 = std::min(npen, p0 + chunk);
    if (p0 < p1) th.emplace_back(work, p0, p1);
  }
  for (auto& t : th) t.join();
  for (int pp = 0; pp < npen; ++pp)
    if (bad[pp]) {
      if (err) *err = "couette: singular pencil matrix at (kx, ky) index (" + std::to_string(pp % Kx) + ", " +
                      std::to_string(pp / Kx) + ")";
      return false;
    }
  return true;
}

namespace {

// Row and column orders of the banded form (couette_setup.h): perm_r[i] / perm_c[i] is the row /
// column of the assembled pencil matrix at position i.
void band_orders(int N, bool mean, std::vector<int>& perm_r, std::vector<int>& perm_c) {
  const int nv = 4 * N + 7;
  perm_r.clear();
  perm_c.clear();
  if (!mean) perm_r.push_back(4 * N + 6);
  perm_c.push_back(4 * N + 6);
  for (int n = 0; n < N; ++n)
    for (int f = 0; f < 4; ++f) {
      perm_r.push_back(f * N + n);
      perm_c.push_back(f * N + n);
    }
  for (int b = 0; b < 6; ++b) {
    perm_r.push_back(4 * N + b);
    perm_c.push_back(4 * N + b);
  }
  if (mean) perm_r.push_back(4 * N + 6);
  (void)nv;
}

// The recombined, reordered pencil matrix A' (row-major nv x nv) and, for the adjoint direction,
// J A'^H J in its place.
void band_matrix(const rbhost::Operators& o, const std::vector<double>& ZS, const std::vector<double>& UP, double al,
                 double be, bool mean, double nu, double a0, bool hermitian, std::vector<cd>& A, std::vector<cd>& B) {
  const int N = o.N, nv = 4 * N + 7;
  assemble_pencil(o, ZS, UP, al, be, mean, nu, cd(a0, 0.0), A);
  auto col_sub = [&](int c, int c2, double w) {  // column c -= w * column c2
    for (int r = 0; r < nv; ++r) A[(size_t)r * nv + c] -= w * A[(size_t)r * nv + c2];
  };
  // ascending j: column j + 2 is still the plain Chebyshev column when column j takes it
  for (int f = 0; f < 3; ++f)
    for (int j = 0; j + 2 < N; ++j) col_sub(f * N + j, f * N + j + 2, 1.0);
  // the pressure columns only where the gauge row reads them (the mean pencil): elsewhere the
  // recombination would raise the condition number of A' by four orders of magnitude
  for (int j = 0; mean && j + 2 < N; j += 2) {
    const double wj = 2.0 / (1.0 - (double)j * j), wj2 = 2.0 / (1.0 - (double)(j + 2) * (j + 2));
    col_sub(3 * N + j, 3 * N + j + 2, wj / wj2);
    // int psi_j dz = 0 exactly; the gauge row's rounding residue is dropped
    A[(size_t)(4 * N + 6) * nv + 3 * N + j] = 0.0;
  }
  std::vector<int> pr, pc;
  band_orders(N, mean, pr, pc);
  B.assign((size_t)nv * nv, cd(0.0, 0.0));
  for (int i = 0; i < nv; ++i)
    for (int k = 0; k < nv; ++k) {
      const cd v = A[(size_t)pr[i] * nv + pc[k]];
      if (!hermitian)
        B[(size_t)i * nv + k] = v;
      else
        B[(size_t)(nv - 1 - k) * nv + (nv - 1 - i)] = std::conj(v);
    }
}

void band_widths(const std::vector<cd>& B, int nv, int& kl, int& ku) {
  kl = ku = 0;
  for (int i = 0; i < nv; ++i)
    for (int k = 0; k < nv; ++k)
      if (B[(size_t)i * nv + k] != 0.0) {
        kl = std::max(kl, i - k);
        ku = std::max(ku, k - i);
      }
}

// Band LU with partial pivoting of B (row-major nv x nv, lower width kl, upper width ku) in place;
// interchanges touch only the columns from j on.  piv[j] = pivot row - j.  False if singular.
bool band_lu(std::vector<cd>& B, int nv, int kl, int ku, std::vector<int>& piv) {
  piv.assign(nv, 0);
  for (int j = 0; j < nv; ++j) {
    const int imax = std::min(nv - 1, j + kl), cmax = std::min(nv - 1, j + kl + ku);
    int p = j;
    double best = std::norm(B[(size_t)j * nv + j]);
    for (int i = j + 1; i <= imax; ++i) {
      const double v = std::norm(B[(size_t)i * nv + j]);
      if (v > best) { best = v; p = i; }
    }
    if (best == 0.0) return false;
    piv[j] = p - j;
    if (p != j)
      for (int c = j; c <= cmax; ++c) std::swap(B[(size_t)j * nv + c], B[(size_t)p * nv + c]);
    const cd inv = 1.0 / B[(size_t)j * nv + j];
    for (int i = j + 1; i <= imax; ++i) {
      const cd l = B[(size_t)i * nv + j] * inv;
      B[(size_t)i * nv + j] = l;
      if (l == 0.0) continue;
      caxpy_sub(&B[(size_t)i * nv + j + 1], &B[(size_t)j * nv + j + 1], l, cmax - j);
    }
  }
  return true;
}

}  // namespace

bool build_band(const rbhost::Operators& o, int Kx, int Ny, double Lx, double Ly, double nu, double a0, int base,
                bool hermitian, BandFactors& F, std::string* err) {
  const int N = o.N, nv = 4 * N + 7, Nyh = Ny / 2, npen = Kx * Nyh;
  std::vector<double> ZS, UP;
  base_flow(o, base, ZS, UP);
  F.ssb.assign((size_t)N * 5, 0.0);
  for (int r = 0; r < N; ++r)
    for (int c = 0; c < N; ++c) {
      const double v = o.SS[(size_t)r * N + c];
      if (v == 0.0) continue;
      if (c < r || c > r + 4) {
        if (err) *err = "couette: the conversion S1S0 is not banded as the banded solve assumes";
        return false;
      }
      F.ssb[(size_t)r * 5 + (c - r)] = v;
    }
  unsigned nt = std::thread::hardware_concurrency();
  if (nt == 0) nt = 1;
  if (nt > 64) nt = 64;
  if ((int)nt > npen) nt = npen;
  const int chunk = (npen + nt - 1) / nt;
  auto pencil = [&](int pp) {
    const int jh = pp / Kx, m = pp % Kx;
    return std::make_tuple(2.0 * M_PI / Lx * m, 2.0 * M_PI / Ly * jh, m == 0 && jh == 0);
  };
  auto run = [&](auto&& body) {
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t) {
      const int p0 = t * chunk, p1 = std::min(npen, p0 + chunk);
      if (p0 < p1) th.emplace_back([&, p0, p1] { body(p0, p1); });
    }
    for (auto& t : th) t.join();
  };
  // pass 1: the band widths (maximum over the pencils)
  std::vector<int> wl(npen, 0), wu(npen, 0);
  run([&](int p0, int p1) {
    std::vector<cd> A, B;
    for (int pp = p0; pp < p1; ++pp) {
      auto [al, be, mean] = pencil(pp);
      band_matrix(o, ZS, UP, al, be, mean, nu, a0, hermitian, A, B);
      band_widths(B, nv, wl[pp], wu[pp]);
    }
  });
  const int kl = *std::max_element(wl.begin(), wl.end()), kus = *std::max_element(wu.begin(), wu.end());
  if (kl > 255) {
    if (err) *err = "couette: banded pencil lower width above 255";
    return false;
  }
  const int kuf = kl + kus;  // U width with the fill of the interchanges
  // pass 2: factorise; U stored at the full width, then trimmed to the widest actual U
  F.nv = nv;
  F.kl = kl;
  F.npen = npen;
  F.L.assign((size_t)npen * nv * kl * 2, 0.0);
  F.U.assign((size_t)npen * nv * kuf * 2, 0.0);
  F.dinv.assign((size_t)npen * nv * 2, 0.0);
  F.piv.assign((size_t)npen * nv, 0);
  std::vector<int> bad(npen, 0), wact(npen, 0);
  run([&](int p0, int p1) {
    std::vector<cd> A, B;
    std::vector<int> piv;
    for (int pp = p0; pp < p1; ++pp) {
      auto [al, be, mean] = pencil(pp);
      band_matrix(o, ZS, UP, al, be, mean, nu, a0, hermitian, A, B);
      if (!band_lu(B, nv, kl, kus, piv)) {
        bad[pp] = 1;
        continue;
      }
      double* Lp = &F.L[(size_t)pp * nv * kl * 2];
      double* Up = &F.U[(size_t)pp * nv * kuf * 2];
      double* Dp = &F.dinv[(size_t)pp * nv * 2];
      for (int j = 0; j < nv; ++j) {
        F.piv[(size_t)pp * nv + j] = (unsigned char)piv[j];
        const cd d = 1.0 / B[(size_t)j * nv + j];
        Dp[2 * j] = d.real();
        Dp[2 * j + 1] = d.imag();
        for (int k = 0; k < kl && j + 1 + k < nv; ++k) {
          const cd l = B[(size_t)(j + 1 + k) * nv + j];
          Lp[((size_t)j * kl + k) * 2] = l.real();
          Lp[((size_t)j * kl + k) * 2 + 1] = l.imag();
        }
      }
      for (int j = 0; j < nv; ++j)
        for (int k = 0; k < kuf && j - 1 - k >= 0; ++k) {
          const int i = j - 1 - k;
          const cd u = B[(size_t)i * nv + j];
          if (u == 0.0) continue;
          wact[pp] = std::max(wact[pp], k + 1);
          const cd us = u / B[(size_t)i * nv + i];
          Up[((size_t)j * kuf + k) * 2] = us.real();
          Up[((size_t)j * kuf + k) * 2 + 1] = us.imag();
        }
    }
  });
  for (int pp = 0; pp < npen; ++pp)
    if (bad[pp]) {
      if (err)
        *err = "couette: singular banded pencil matrix at (kx, ky) index (" + std::to_string(pp % Kx) + ", " +
               std::to_string(pp / Kx) + ")";
      return false;
    }
  const int ku = std::max(1, *std::max_element(wact.begin(), wact.end()));
  if (ku < kuf) {  // trim every U row to the widest actual one (in place: rows only move down)
    for (size_t r = 0; r < (size_t)npen * nv; ++r)
      for (int k = 0; k < ku; ++k) {
        F.U[(r * ku + k) * 2] = F.U[(r * kuf + k) * 2];
        F.U[(r * ku + k) * 2 + 1] = F.U[(r * kuf + k) * 2 + 1];
      }
    F.U.resize((size_t)npen * nv * ku * 2);
  }
  F.ku = ku;
  return true;
}

bool band_solve_host(const rbhost::Operators& o, double al, double be, double nu, double a0, int base, bool transpose,
                     const cd* in, cd* out, std::string* err) {
  const int N = o.N, nv = 4 * N + 7;
  const bool mean = al == 0.0 && be == 0.0;
  std::vector<double> ZS, UP;
  base_flow(o, base, ZS, UP);
  std::vector<cd> A, B;
  band_matrix(o, ZS, UP, al, be, mean, nu, a0, transpose, A, B);
  int kl = 0, ku = 0;
  band_widths(B, nv, kl, ku);
  std::vector<int> piv;
  if (!band_lu(B, nv, kl, ku, piv)) {
    if (err) *err = "couette: singular banded pencil matrix";
    return false;
  }
  std::vector<double> ssb((size_t)N * 5, 0.0);
  for (int r = 0; r < N; ++r)
    for (int d = 0; d < 5 && r + d < N; ++d) ssb[(size_t)r * 5 + d] = o.SS[(size_t)r * N + r + d];
  std::vector<cd> y(nv, cd(0.0, 0.0));
  const int o_rows = mean ? 0 : 1;  // position of mode 0's momentum rows in A'
  for (int f = 0; f < 3; ++f)
    for (int n = 0; n < N; ++n) {
      if (!transpose) {
        cd b = 0.0;
        for (int d = 0; d < 5 && n + d < N; ++d) b += ssb[(size_t)n * 5 + d] * in[f * N + n + d];
        y[o_rows + 4 * n + f] = b;
      } else {
        y[nv - 1 - (1 + 4 * n + f)] = in[f * N + n] - (n + 2 < N ? in[f * N + n + 2] : cd(0.0, 0.0));
      }
    }
  // the sweeps of the GPU kernel: interchange and multipliers, 1/U_jj, row-scaled U by columns
  for (int j = 0; j < nv; ++j) {
    if (piv[j]) std::swap(y[j], y[j + piv[j]]);
    for (int i = j + 1; i <= std::min(nv - 1, j + kl); ++i) y[i] -= B[(size_t)i * nv + j] * y[j];
  }
  for (int j = 0; j < nv; ++j) y[j] *= 1.0 / B[(size_t)j * nv + j];
  for (int j = nv - 1; j >= 0; --j)
    for (int i = std::max(0, j - kl - ku); i < j; ++i)
      y[i] -= (B[(size_t)i * nv + j] / B[(size_t)i * nv + i]) * y[j];
  for (int f = 0; f < 3; ++f)
    for (int n = 0; n < N; ++n) {
      if (!transpose) {
        out[f * N + n] = y[1 + 4 * n + f] - (n >= 2 ? y[1 + 4 * (n - 2) + f] : cd(0.0, 0.0));
      } else {
        cd v = 0.0;
        for (int d = 0; d < 5 && n - d >= 0; ++d) v += ssb[(size_t)(n - d) * 5 + d] * y[nv - 1 - (o_rows + 4 * (n - d) + f)];
        out[f * N + n] = v;
      }
    }
  return true;
}

bool build_evp(const rbhost::Operators& o, int base, int P, const double* prm, const double* shift,
               std::vector<double>& T, std::vector<double>& RH, std::string* err) {
  const int N = o.N, nv = 4 * N + 7, H = 3 * N;
  std::vector<double> Um, UP;
  base_flow(o, base, Um, UP);
  const size_t per = (size_t)nv * H * 2;
  T.assign((size_t)P * per, 0.0);
  RH.assign((size_t)P * per, 0.0);
  std::vector<int> bad(P, 0);
  auto work = [&](int p0, int p1) {
    std::vector<cd> A, B;
    std::vector<int> piv;
    for (int pp = p0; pp < p1; ++pp) {
      const double al = prm[3 * pp], be = prm[3 * pp + 1], Re = prm[3 * pp + 2];
      const cd sigma(shift[2 * pp], shift[2 * pp + 1]);
      assemble_pencil(o, Um, UP, al, be, al == 0.0 && be == 0.0, 1.0 / Re, sigma, A);
      if (!lu_factor(A, piv, nv)) {
        bad[pp] = 1;
        continue;
      }
      B.assign((size_t)nv * H, cd(0.0, 0.0));
      for (int f = 0; f < 3; ++f)
        for (int c = 0; c < N; ++c)
          for (int r = 0; r < N; ++r) B[(size_t)(f * N + r) * H + f * N + c] = o.SS[r * N + c];
      lu_solve_multi(A, piv, nv, B, H);
      double* t = &T[(size_t)pp * per];
      for (size_t i = 0; i < (size_t)nv * H; ++i) { t[2 * i] = B[i].real(); t[2 * i + 1] = B[i].imag(); }
      B.assign((size_t)nv * H, cd(0.0, 0.0));
      for (int r = 0; r < H; ++r) B[(size_t)r * H + r] = 1.0;
      lu_solve_h_multi(A, piv, nv, B, H);
      double* rh = &RH[(size_t)pp * per];
      for (size_t i = 0; i < (size_t)nv * H; ++i) { rh[2 * i] = B[i].real(); rh[2 * i + 1] = B[i].imag(); }
    }
  };
  unsigned nt = std::thread::hardware_concurrency();
  if (nt == 0) nt = 1;
  if (nt > 64) nt = 64;
  if ((int)nt > P) nt = P;
  std::vector<std::thread> th;
  const int chunk = (P + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    const int p0 = t * chunk, p1 = std::min(P, p0 + chunk);
    if (p0 < p1) th.emplace_back(work, p0, p1);
  }
  for (auto& t : th) t.join();
  for (int pp = 0; pp < P; ++pp)
    if (bad[pp]) {
      if (err) *err = "eigen: singular shifted pencil matrix at pencil " + std::to_string(pp);
      return false;
    }
  return true;
}

}  // namespace couhost
}  // namespace spadj
