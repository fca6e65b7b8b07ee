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

// Complex Phi = [(a0 M + L)^-1]_{prognostic} * blockdiag(S1S0) (3N x 3N) for every pencil
// (a0 real for the timestep operators, a0 = i omega for the resolvent at frequency omega)
// (kx index m = 0..Kx-1, ky index jh = 0..Ny/2-1, ky = jh >= 0), stored twice as interleaved
// (re, im) doubles: phiF[jh][m][k][r] = Phi[r][k] and phiA[jh][m][r][k] = Phi[r][k].
// Pencils with ky < 0 follow from Phi(kx, -ky) = D Phi(kx, ky) D, D = diag(1, -1, 1) on
// (u, v, w).  Returns false (and sets err) if a pencil matrix is singular.
bool build_phi(const rbhost::Operators& o, int Kx, int Ny, double Lx, double Ly, double nu, std::complex<double> a0,
               std::vector<double>& phiF, std::vector<double>& phiA, std::string* err);

}  // namespace couhost
}  // namespace spadj
