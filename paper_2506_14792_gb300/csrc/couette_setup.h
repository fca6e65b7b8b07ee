// Host construction of the plane-Couette pencil solution operators (couette_setup.cpp).
//
// Pencil variable ordering: [u_0..u_{N-1}, v_*, w_*, p_*, tau_u1, tau_u2, tau_v1, tau_v2,
// tau_w1, tau_w2, tau_p]; equation rows: [u-eq (C^(2)), v-eq, w-eq, continuity (C^(1)),
// u(-1), u(1), v(-1), v(1), w(-1), w(1), gauge].
#pragma once
#include <complex>
#include <string>
#include <vector>

#include "rb_setup.h"

namespace spadj {
namespace couhost {

using cd = std::complex<double>;

// Complex LU with partial pivoting of the row-major n x n matrix a, in place (P A = L U with
// unit L); piv[k] is the row swapped with row k at step k.  False if a pivot is exactly 0.
bool lu_factor(std::vector<cd>& a, std::vector<int>& piv, int n);
// Solve A X = B (nr right-hand sides, B row-major n x nr, overwritten) with those factors.
void lu_solve_multi(const std::vector<cd>& a, const std::vector<int>& piv, int n, std::vector<cd>& B, int nr);
// Solve A^H X = B with the same factors (the adjoint solve reuses the forward factorisation).
void lu_solve_h_multi(const std::vector<cd>& a, const std::vector<int>& piv, int n, std::vector<cd>& B, int nr);

// Base-flow matrices on N modes (row-major N x N, C^(2) rows acting on T coefficients):
// Umat = [U T_n], UPmat = [U' T_n], the products formed exactly in the T basis, converted with
// S1 S0 and truncated; base 0: plane Couette U = z; base 1: plane Poiseuille U = 1 - z^2.
void base_flow(const rbhost::Operators& o, int base, std::vector<double>& Umat, std::vector<double>& UPmat);

// a0 M + L of the pencil (alpha, beta) at viscosity nu for the base flow (Umat, UPmat), row-major
// (4N + 7) x (4N + 7); mean selects the gauge rows of the (0, 0) pencil.
void assemble_pencil(const rbhost::Operators& o, const std::vector<double>& Umat, const std::vector<double>& UPmat,
                     double al, double be, bool mean, double nu, cd a0, std::vector<cd>& A);

// Complex Phi = [(a0 M + L)^-1]_{prognostic} * blockdiag(S1S0) (3N x 3N) for every pencil
// (a0 real for the timestep operators, a0 = i omega for the resolvent at frequency omega)
// (kx index m = 0..Kx-1, ky index jh = 0..Ny/2-1, ky = jh >= 0), stored twice as interleaved
// (re, im) doubles: phiF[jh][m][k][r] = Phi[r][k] and phiA[jh][m][r][k] = Phi[r][k].
// Pencils with ky < 0 follow from Phi(kx, -ky) = D Phi(kx, ky) D, D = diag(1, -1, 1) on
// (u, v, w).  Returns false (and sets err) if a pencil matrix is singular.
// base selects the laminar profile as in base_flow (0 plane Couette, 1 plane Poiseuille).
bool build_phi(const rbhost::Operators& o, int Kx, int Ny, double Lx, double Ly, double nu, std::complex<double> a0,
               std::vector<double>& phiF, std::vector<double>& phiA, std::string* err, int base = 0);

// Banded factors of the step solves (the alternative to the dense Phi; same linear map up to
// rounding).  The pencil matrix A = a0 M + L is right-preconditioned by a recombination R of the
// Chebyshev columns (velocity: phi_j = T_j - T_{j+2} for j <= N-3, which vanish at z = +-1; on
// the mean pencil also pressure: psi_j = T_j - (int T_j / int T_{j+2}) T_{j+2} for even j <= N-3,
// which integrate to zero), so the boundary rows and the gauge row touch only the last two
// modes; rows and columns
// are then ordered by Chebyshev mode (the four equations / variables of a mode together), with
//   rows    [gauge, modes 0..N-1 (u-eq, v-eq, w-eq, continuity), u(-1), u(1), v(-1), v(1), w(-1), w(1)]
//           (the mean pencil puts the gauge row last),
//   columns [tau_p, modes 0..N-1 (u, v, w, p), tau_u1, tau_u2, tau_v1, tau_v2, tau_w1, tau_w2],
// which makes A' = Pr A R Pc^T banded (kl = 12, ku = 20 at N = 64).  A' is factorised by band
// LU with partial pivoting (row interchanges confined to the band, LAPACK's band convention:
// the multipliers of column j are not moved by later interchanges).  The adjoint direction
// factorises J A'^H J (J the order reversal, so its lower band is A's and the forward sweep of
// both directions is the short one) instead of reusing A's factors transposed: the same
// operator A^-H, with the solve in the same column-oriented form.
// Solve semantics of one factor set (n = nv unknowns), as the GPU kernel runs it:
//   for j = 0..n-1: y_j <-> y_{j + piv[j]}; y_{j+1+k} -= L[j][k] y_j (k < kl)
//   y_j *= dinv[j]
//   for j = n-1..0: y_{j-1-k} -= U[j][k] y_j (k < ku)
// with dinv[j] = 1 / U_jj and U[j][k] = U_{j-1-k, j} / U_{j-1-k, j-1-k} (the rows of U scaled to a
// unit diagonal, so the back sweep needs no division).
struct BandFactors {
  int nv = 0, kl = 0, ku = 0, npen = 0;
  std::vector<double> L;           // [pencil][j][kl] complex, interleaved (re, im)
  std::vector<double> U;           // [pencil][j][ku] complex
  std::vector<double> dinv;        // [pencil][j] complex
  std::vector<unsigned char> piv;  // [pencil][j]: pivot row - j (0..kl)
  std::vector<double> ssb;         // [N][5]: S1S0[n][n + d] (the conversion's band)
};

// The banded factors of every pencil (pencil index jh * Kx + m, ky = jh >= 0, as build_phi) at
// a0 (real); hermitian selects the adjoint direction.  False (and err) if a pencil is singular,
// the conversion S1S0 is not banded as assumed, or kl exceeds 255.
bool build_band(const rbhost::Operators& o, int Kx, int Ny, double Lx, double Ly, double nu, double a0, int base,
                bool hermitian, BandFactors& F, std::string* err);

// One pencil's banded solve on the host with the arithmetic of the GPU kernel (test support):
// x = [A'^-1 (S1S0 v on the momentum rows)] recombined to the prognostic coefficients (transpose = 0),
// or v = S1S0^T [momentum rows of (J A'^H J)^-1 J (R^T x)] (transpose = 1), for the pencil
// (alpha, beta) at a0 (real); v, x: 3N complex (u, v, w coefficients), the ky >= 0 member (no
// projection).  False (and err) if the pencil is singular.
bool band_solve_host(const rbhost::Operators& o, double al, double be, double nu, double a0, int base, bool transpose,
                     const std::complex<double>* in, std::complex<double>* out, std::string* err);

// Shift-invert operators of P eigenvalue pencils (prm[p] = alpha, beta, Re; shift[p] = sigma as
// (re, im)) of the base flow `base`: with A_p = sigma_p M + L_p (one LU per pencil),
//   T[p]  = A_p^-1 [S1S0 on the u, v, w momentum rows]   ((4N + 7) x 3N),
//   RH[p] = A_p^-H [e_0 .. e_{3N-1}]                      ((4N + 7) x 3N),
// both row-major with interleaved (re, im); RH by the adjoint solve with the same factors.
// The first 3N rows of T are the prognostic shift-invert operator Phi(sigma), and row i of RH
// holds conj((A^-1)[r][i]) for r < 3N.  Returns false (and sets err) if a pencil is singular.
bool build_evp(const rbhost::Operators& o, int base, int P, const double* prm, const double* shift,
               std::vector<double>& T, std::vector<double>& RH, std::string* err);

}  // namespace couhost
}  // namespace spadj
