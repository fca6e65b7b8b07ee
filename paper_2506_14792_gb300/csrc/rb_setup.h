// Host construction of the Chebyshev/ultraspherical operators (shared by the Rayleigh-Benard
// and plane-Couette pencils) and of the Rayleigh-Benard solution operators (rb_setup.cpp).
//
// Pencil variable ordering: [u_0..u_{N-1}, w_*, theta_*, p_*, tau_u1, tau_u2, tau_w1,
// tau_w2, tau_t1, tau_t2, tau_p]; equation rows: [u-eq (C^(2)), w-eq, theta-eq,
// continuity (C^(1)), u(z=0), u(z=1), w(0), w(1), theta(0), theta(1), gauge].
#pragma once
#include <string>
#include <vector>

namespace spadj {
namespace rbhost {

struct Operators {
  int N = 0, Mz = 0;
  std::vector<double> SS, DD, SD, S0, D0;  // N x N, row-major (z-scaled derivatives)
  std::vector<double> Dz;                  // N x N derivative in the T basis
  std::vector<double> Cz, Cdz;             // Mz x N: T_n(xi_j), dT_n/dz(xi_j)
  std::vector<double> Gz;                  // N x Mz: (w_n / Mz) T_n(xi_j)
  std::vector<double> G;                   // N x N: int_0^1 T_m T_n dz
  int lift_row = 0;
  double lift_val = 0.0;
};

// zs = d xi / dz: 2 for z in [0, 1] (Rayleigh-Benard), 1 for z in [-1, 1] (plane Couette).
Operators build_operators(int N, int Mz, double zs = 2.0);

// Ultraspherical building blocks on N modes (row-major N x N, derivatives scaled by s).
std::vector<double> op_D0(int N, double s);
std::vector<double> op_D1(int N, double s);
std::vector<double> op_S0(int N);
std::vector<double> op_S1(int N);
std::vector<double> matmul(const std::vector<double>& a, const std::vector<double>& b, int N);

// Phi' for every pencil m = 0..Kx-1 (layout [m][3N][3N], row-major), for the implicit
// matrix M + b L.  Returns false (and sets err) if a pencil matrix is singular.
bool build_phi(const Operators& o, int Kx, double Lx, double nu, double kappa, double b, std::vector<double>& phi,
               std::string* err);

}  // namespace rbhost
}  // namespace spadj
