// 3D plane Couette flow: SBDF1 -> SBDF2 IMEX forward step, tangent step and exact discrete
// adjoint on the GPU, with binomial checkpointing for the energy-gain gradient.
//
// Per step n (eq. imex with M = S1S0 on the prognostic rows and b_i = 0 for i >= 1):
//   f_{n-1} = F(x_{n-1});   v = sum_i (c_i f_{n-i} - a_i x_{n-i});   x_n = P Phi_n v
// with Phi_n the per-pencil prognostic solution operator of (a_0 M + L) (couette_setup.cpp;
// SBDF1 for n = 1, SBDF2 after) and P the projection onto admissible coefficients.
// Reverse (eq. IMEX_adjoint in prognostic form, W_n = Phi_n^H P xbar_n):
//   xbar_k = src_k + (dF/dx)(x_k)^H (c_1^{k+1} W_{k+1} + c_2^{k+2} W_{k+2})
//            - a_1^{k+1} W_{k+1} - a_2^{k+2} W_{k+2},
// with the coefficients of step k+i multiplying W_{k+i}, and dJ/dX_0 = xbar_0 (no solve).
// F = u x omega is evaluated pseudospectrally: z transforms (Chebyshev matrices with
// reflection folding), y FFTs over column tiles, x FFTs per row, grid products formed inside
// the x-forward FFT (Sparse spectral methods section).
#include <cmath>
#include <string>
#include <vector>

#include "couette_kernels.cuh"
#include "couette_setup.h"
#include "problem.h"
#include "rb_kernels.cuh"
#include "revolve.h"

namespace spadj {
namespace {

using namespace rbk;
using namespace couk;

struct Couette : EqImpl {
  int Nx = 0, Ny = 0, N = 0, Kx = 0, Mx = 0, My = 0, Mz = 0, L = 0, P = 0, order = 2;
  int base = 0;  // laminar profile: 0 plane Couette U = z, 1 plane Poiseuille U = 1 - z^2
  double Lx = 0, Ly = 0, Re = 0, nu = 0, dt = 0;
  int nonlinear = 1;
  size_t nfield = 0;  // complex entries of one field [Ny][Kx][N]
  size_t ns = 0;      // complex entries of a state [3][Ny][Kx][N]
  size_t nzm = 0;     // complex entries of a z-mixed array [Mz][Ny][Kx]
  size_t nym = 0;     // complex entries of a y-mixed array [Mz][My][Kx]
  size_t npts = 0;    // grid points Mz*My*Mx
  XParams xp{};
  YParams yp{};
  DevBuf wmx, w2y, czE, cdzE, gzF, gzTE, czTF, cdzTF, gmat, phi1F, phi1A, phi2F, phi2A, one;
  // banded factors of the step solves: [scheme order - 1][0 forward, 1 adjoint]
  struct BandDev {
    DevBuf L, U, dinv, piv, ssb;
    int kl = 0, ku = 0, nv = 0;
  };
  BandDev band[2][2];
  bool band_ok = false, dense_ok = false, band_too_wide = false;
  bool band_auto = true;  // the form option 12 = -1 selects: banded when the pencil pairs fill the GPU
  DevBuf Zm, Ym, Gf, dGf, Gb, Fg, Xr, Fr, dXr, dFr, Wr, xbar, src0, partial, edev, sdev, Jdev, slots, wts;
  DevBuf phiRF, phiRA, ginv, nrm, g2;  // resolvent operators of the last frequency, G^-1, per-pencil norms
  DevBuf htraj, hdtraj, dWr, dxbar, htmp;  // Hessian-vector product: trajectories and second-order cotangents
  HostBuf hslots;  // host tier of the two-level checkpoint schedule
  double res_omega = 0.0;
  bool res_built = false;
  size_t zsmem = 0, xsmem = 0, ysmem = 0;
  rbhost::Operators ops;
  int xnb = 1;  // x-FFT launch variant, xvar(rows per CTA, threads) (tuned at creation)

  size_t state_len(int which) const override {
    if (which == 0) return 2 * ns;
    if (which == 1) return npts;
    if (which == 3) return 2 * nfield;
    return 0;
  }

  double2* st(DevBuf& b, int i) { return b.as<double2>() + (size_t)i * ns; }
  double2* zm(int i) { return Zm.as<double2>() + (size_t)i * nzm; }
  double2* ym(int i) { return Ym.as<double2>() + (size_t)i * nym; }
  double* grid(DevBuf& b, int i) { return b.as<double>() + (size_t)i * npts; }
  static double2* fld(double2* s, size_t nf, int q) { return s + (size_t)q * nf; }

  spadj_status init(Problem* p) {
    const spadj_desc& d = p->desc;
    Nx = d.n[0];
    Ny = d.n[1];
    N = d.n[2];
    if (Nx < 4 || Nx % 4 != 0 || Ny < 4 || Ny % 2 != 0 || N < 8 || N % 4 != 0)
      return p->fail(SPADJ_ERR_INVALID,
                     "couette: n[0] must be a multiple of 4, n[1] even (>= 4), n[2] a multiple of 4 (>= 8)");
    if (N > 128) return p->fail(SPADJ_ERR_INVALID, "couette: n[2] must be <= 128");
    if (d.scheme != SPADJ_SBDF2 && d.scheme != SPADJ_SBDF1)
      return p->fail(SPADJ_ERR_UNSUPPORTED, "couette: scheme must be SBDF1 or SBDF2");
    if (d.batch != 1) return p->fail(SPADJ_ERR_UNSUPPORTED, "couette: batch must be 1");
    order = d.scheme == SPADJ_SBDF1 ? 1 : 2;
    Re = d.params[0];
    if (!(Re > 0)) return p->fail(SPADJ_ERR_INVALID, "couette: params[0] (Reynolds number) must be > 0");
    nu = 1.0 / Re;
    base = (int)d.params[1];
    if ((base != 0 && base != 1) || (double)base != d.params[1])
      return p->fail(SPADJ_ERR_INVALID, "couette: params[1] must be 0 (plane Couette) or 1 (plane Poiseuille)");
    dt = d.dt;
    nonlinear = d.nonlinear;
    Lx = d.length[0] > 0 ? d.length[0] : 4.0 * M_PI;
    Ly = d.length[1] > 0 ? d.length[1] : 2.0 * M_PI;
    Kx = Nx / 2;
    Mx = 3 * Nx / 2;
    My = 3 * Ny / 2;
    Mz = 3 * N / 2;
    L = Mx / 2;
    P = Ny * Kx;
    nfield = (size_t)P * N;
    ns = 3 * nfield;
    nzm = (size_t)Mz * P;
    nym = (size_t)Mz * My * Kx;
    npts = (size_t)Mz * My * Mx;
    xp.Kx = Kx; xp.Mx = Mx; xp.L = L; xp.kscale = 2.0 * M_PI / Lx;
    xp.plan = make_plan(L);
    yp.Kx = Kx; yp.Ny = Ny; yp.My = My;
    yp.TK = Kx < 8 ? Kx : 8;
    yp.ntile = (Kx + yp.TK - 1) / yp.TK;
    yp.kxs = 2.0 * M_PI / Lx; yp.kys = 2.0 * M_PI / Ly;
    yp.plan = make_plan(My);
    if (xp.plan.nrad < 0 || yp.plan.nrad < 0)
      return p->fail(SPADJ_ERR_INVALID, "couette: 3*n[0]/4 and 3*n[1]/2 must be of the form 2^a 3^b");

    rbhost::Operators o = rbhost::build_operators(N, Mz, 1.0);
    ops = o;
    const int Mh = Mz / 2;
    std::vector<double> hczE((size_t)Mh * N), hcdzE((size_t)Mh * N), hgzF((size_t)N * Mh), hgzTE((size_t)Mh * N),
        hczTF((size_t)N * Mh), hcdzTF((size_t)N * Mh);
    for (int j = 0; j < Mh; ++j)
      for (int n = 0; n < N; ++n) {
        hczE[(size_t)j * N + n] = o.Cz[(size_t)j * N + n];
        hcdzE[(size_t)j * N + n] = o.Cdz[(size_t)j * N + n];
        hgzTE[(size_t)j * N + n] = o.Gz[(size_t)n * Mz + j];
        hgzF[(size_t)n * Mh + j] = o.Gz[(size_t)n * Mz + j];
        hczTF[(size_t)n * Mh + j] = o.Cz[(size_t)j * N + n];
        hcdzTF[(size_t)n * Mh + j] = o.Cdz[(size_t)j * N + n];
      }
    std::vector<double2> hwx(Mx), hwy(2 * My);
    for (int m = 0; m < Mx; ++m) {
      const double th = -2.0 * M_PI * (double)m / (double)Mx;
      hwx[m] = make_double2(std::cos(th), std::sin(th));
    }
    for (int m = 0; m < 2 * My; ++m) {
      const double th = -2.0 * M_PI * (double)m / (double)(2 * My);
      hwy[m] = make_double2(std::cos(th), std::sin(th));
    }
    {  // the butterflies' scaled-twiddle records follow each twiddle table in its buffer
      const std::vector<double2> sx = scaled_twiddle_table(xp.plan), sy = scaled_twiddle_table(yp.plan);
      hwx.insert(hwx.end(), sx.begin(), sx.end());
      hwy.insert(hwy.end(), sy.begin(), sy.end());
    }
    const double hone = 1.0;
    auto up = [&](DevBuf& b, const void* h, size_t bytes) -> cudaError_t {
      cudaError_t e = b.ensure(bytes);
      if (e != cudaSuccess) return e;
      return cudaMemcpyAsync(b.ptr, h, bytes, cudaMemcpyHostToDevice, p->stream);
    };
    SPADJ_CUDA_TRY(p, up(wmx, hwx.data(), sizeof(double2) * hwx.size()));
    SPADJ_CUDA_TRY(p, up(w2y, hwy.data(), sizeof(double2) * hwy.size()));
    SPADJ_CUDA_TRY(p, up(czE, hczE.data(), sizeof(double) * hczE.size()));
    SPADJ_CUDA_TRY(p, up(cdzE, hcdzE.data(), sizeof(double) * hcdzE.size()));
    SPADJ_CUDA_TRY(p, up(gzF, hgzF.data(), sizeof(double) * hgzF.size()));
    SPADJ_CUDA_TRY(p, up(gzTE, hgzTE.data(), sizeof(double) * hgzTE.size()));
    SPADJ_CUDA_TRY(p, up(czTF, hczTF.data(), sizeof(double) * hczTF.size()));
    SPADJ_CUDA_TRY(p, up(cdzTF, hcdzTF.data(), sizeof(double) * hcdzTF.size()));
    SPADJ_CUDA_TRY(p, up(gmat, o.G.data(), sizeof(double) * o.G.size()));
    SPADJ_CUDA_TRY(p, up(one, &hone, sizeof(double)));
    SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    xp.WM = wmx.as<double2>();
    yp.W2 = w2y.as<double2>();
    bind_scaled_twiddles(xp.plan, xp.WM + Mx);
    bind_scaled_twiddles(yp.plan, yp.W2 + 2 * My);
    const size_t sb = sizeof(double2) * ns, gb = sizeof(double) * npts;
    SPADJ_CUDA_TRY(p, Zm.ensure(6 * sizeof(double2) * nzm));
    SPADJ_CUDA_TRY(p, Ym.ensure(6 * sizeof(double2) * nym));
    SPADJ_CUDA_TRY(p, Gf.ensure(6 * gb));
    SPADJ_CUDA_TRY(p, dGf.ensure(6 * gb));
    SPADJ_CUDA_TRY(p, Gb.ensure(6 * gb));
    SPADJ_CUDA_TRY(p, Fg.ensure(3 * gb));
    SPADJ_CUDA_TRY(p, Xr.ensure(3 * sb));
    SPADJ_CUDA_TRY(p, Fr.ensure(2 * sb));
    SPADJ_CUDA_TRY(p, Wr.ensure(3 * sb));
    SPADJ_CUDA_TRY(p, xbar.ensure(sb));
    SPADJ_CUDA_TRY(p, src0.ensure(sb));
    SPADJ_CUDA_TRY(p, partial.ensure(sizeof(double) * P));
    SPADJ_CUDA_TRY(p, edev.ensure(sizeof(double) * 2));
    SPADJ_CUDA_TRY(p, sdev.ensure(sizeof(double) * 2));
    SPADJ_CUDA_TRY(p, Jdev.ensure(sizeof(double)));
    zsmem = (size_t)2 * 2 * (size_t)std::max(N, Mz / 2) * kTM * sizeof(double2);
    xsmem = sizeof(double2) * (4 * L + Kx);
    ysmem = sizeof(double2) * 2 * (size_t)My * yp.TK;
    {  // the step-solve operators of the selected form (the other one is built on first use)
      // One warp per pencil pair runs the band sweeps: with fewer than 8 pairs per SM the warps
      // cannot keep the FP64 pipe busy and the dense Phi (a CTA per pair) is faster (measured:
      // 2112 pairs on 152 SMs 2.3x faster banded, 544 pairs 2x slower).
      int dev = 0, sms = 0;
      SPADJ_CUDA_TRY(p, cudaGetDevice(&dev));
      SPADJ_CUDA_TRY(p, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      band_auto = (long long)Kx * (Ny / 2 + 1) >= 8LL * sms;
      spadj_status s = use_band(p) ? ensure_band(p) : ensure_dense(p);
      if (s != SPADJ_OK) return s;
    }
    {  // x-FFT rows per CTA, timed on the six inverse transforms of one F evaluation
      SPADJ_CUDA_TRY(p, cudaMemsetAsync(Ym.ptr, 0, Ym.bytes, p->stream));
      XJobs xj{};
      for (int q = 0; q < 6; ++q) xj.j[q] = xc2r(ym(q), 1.0, 1.0, grid(Gf, q));
      xj.n = 6;
      cudaError_t e = cudaSuccess;
      xnb = tune_xfft_rows(xj, xp, Mz * My, p->stream, p->x_rows, &e);
      SPADJ_CUDA_TRY(p, e);
    }
    return SPADJ_OK;
  }

  // ---- launches ------------------------------------------------------------------------------
  ZJobs zjobs(int expand) {
    ZJobs js{};
    js.expand = expand;
    js.ncols = P;
    js.kxn = Kx;
    js.nyk = Ny;
    js.kxs = 2.0 * M_PI / Lx;
    js.kys = 2.0 * M_PI / Ly;
    return js;
  }
  ZJob zexp(const double2* in, const double* mat, int deriv, double2* out) {
    ZJob j{};
    j.in[0] = in; j.mat[0] = mat; j.alpha[0] = 1.0; j.deriv[0] = deriv; j.nterm = 1;
    j.out = out; j.I = Mz; j.K = N; j.ik = 1; j.im = N; j.oi = P; j.om = 1;
    return j;
  }
  ZJob zfld(const double2* in, const double* mat, int deriv, double2* out) {
    ZJob j{};
    j.in[0] = in; j.mat[0] = mat; j.alpha[0] = 1.0; j.deriv[0] = deriv; j.nterm = 1;
    j.out = out; j.I = N; j.K = Mz; j.ik = P; j.im = 1; j.oi = 1; j.om = N;
    return j;
  }
  spadj_status launch_z(Problem* p, ZJobs& js) {
    double f = 0;
    for (int i = 0; i < js.n; ++i) f += 4.0 * P * N * (Mz / 2) * js.j[i].nterm;
    const int threads = zmm_threads(js.expand, js.j[0].I);
    cudaEvent_t t = p->tic();
    SPADJ_CUDA_TRY(p, launch_kernel(p->pdl, zmm_kernel, dim3(P, js.n), dim3(threads), zsmem, p->stream, js));
    p->toc(t, KC_ZTRANSFORM, f);
    return check_launch(p, "couette zmm");
  }
  YJob yinv(double2* out, double scale) {
    YJob j{};
    j.dir = 0; j.out = out; j.scale = scale;
    return j;
  }
  static void yadd(YJob& j, const double2* in, double alpha, int mult) {
    j.in[j.nin] = in; j.alpha[j.nin] = alpha; j.mult[j.nin] = mult; ++j.nin;
  }
  YJob yfwd(const double2* in, double scale, double2* out) {
    YJob j{};
    j.dir = 1; j.in[0] = in; j.alpha[0] = 1.0; j.nin = 1; j.scale = scale; j.out = out;
    return j;
  }
  spadj_status launch_y(Problem* p, YJobs& js) {
    const double f = js.n * (double)Mz * Kx * 5.0 * My * std::log2((double)My);
    cudaEvent_t t = p->tic();
    SPADJ_CUDA_TRY(p, launch_kernel(p->pdl, yfft_kernel, dim3(Mz * yp.ntile, js.n), dim3(128), ysmem, p->stream, js, yp));
    p->toc(t, KC_YFFT, f);
    return check_launch(p, "couette yfft");
  }
  XJob xc2r(const double2* in, double w0, double w, double* out) {
    XJob j{};
    j.dir = 0; j.cin = in; j.w0 = w0; j.w = w; j.rout = out;
    return j;
  }
  XJob xr2c(const double* in, double s0, double s, double2* out) {
    XJob j{};
    j.dir = 1; j.rin[0] = in; j.nr = 1; j.s0 = s0; j.s = s; j.cout = out;
    return j;
  }
  spadj_status launch_x(Problem* p, XJobs& js) {
    const double f = js.n * (double)Mz * My * 2.5 * Mx * std::log2((double)Mx);
    cudaEvent_t t = p->tic();
    SPADJ_CUDA_TRY(p, launch_xfft(p->pdl, p->x_rows ? p->x_rows : xnb, js, xp, Mz * My, p->stream));
    p->toc(t, KC_XFFT, f);
    return check_launch(p, "couette xfft");
  }

  // grid fields (slots 0 u, 1 v, 2 w, 3 omega_x, 4 omega_y, 5 omega_z) of the state x into G
  spadj_status c2g6(Problem* p, const double2* x, DevBuf& G) {
    ZJobs zj = zjobs(1);
    zj.j[0] = zexp(fld(const_cast<double2*>(x), nfield, 0), czE.as<double>(), 0, zm(0));
    zj.j[1] = zexp(fld(const_cast<double2*>(x), nfield, 1), czE.as<double>(), 0, zm(1));
    zj.j[2] = zexp(fld(const_cast<double2*>(x), nfield, 2), czE.as<double>(), 0, zm(2));
    zj.j[3] = zexp(fld(const_cast<double2*>(x), nfield, 0), cdzE.as<double>(), 1, zm(3));  // dz u
    zj.j[4] = zexp(fld(const_cast<double2*>(x), nfield, 1), cdzE.as<double>(), 1, zm(4));  // dz v
    zj.n = 5;
    spadj_status s = launch_z(p, zj);
    if (s != SPADJ_OK) return s;
    YJobs yj{};
    for (int q = 0; q < 6; ++q) yj.j[q] = yinv(ym(q), 1.0);
    yadd(yj.j[0], zm(0), 1.0, 0);
    yadd(yj.j[1], zm(1), 1.0, 0);
    yadd(yj.j[2], zm(2), 1.0, 0);
    yadd(yj.j[3], zm(2), 1.0, 2); yadd(yj.j[3], zm(4), -1.0, 0);  // omega_x = i ky w - dz v
    yadd(yj.j[4], zm(3), 1.0, 0); yadd(yj.j[4], zm(2), -1.0, 1);  // omega_y = dz u - i kx w
    yadd(yj.j[5], zm(1), 1.0, 1); yadd(yj.j[5], zm(0), -1.0, 2);  // omega_z = i kx v - i ky u
    yj.n = 6;
    if ((s = launch_y(p, yj)) != SPADJ_OK) return s;
    XJobs xj{};
    for (int q = 0; q < 6; ++q) xj.j[q] = xc2r(ym(q), 1.0, 1.0, grid(G, q));
    xj.n = 6;
    return launch_x(p, xj);
  }

  // F = u x omega (or its tangent when dGp is non-null) from the grid fields -> T-space f
  spadj_status g2c3(Problem* p, double2* f, const double* Gp, const double* dGp) {
    static const int pa[3][2] = {{1, 2}, {2, 0}, {0, 1}};
    static const int pb[3][2] = {{5, 4}, {3, 5}, {4, 3}};
    XJobs xj{};
    for (int q = 0; q < 3; ++q) {
      XJob j = xr2c(nullptr, 1.0 / Mx, 1.0 / Mx, ym(q));
      j.nprod = 2;
      j.pa[0] = pa[q][0]; j.pb[0] = pb[q][0]; j.ps[0] = 1.0;
      j.pa[1] = pa[q][1]; j.pb[1] = pb[q][1]; j.ps[1] = -1.0;
      j.G = Gp; j.dG = dGp; j.npts = (int)npts;
      xj.j[q] = j;
    }
    xj.n = 3;
    spadj_status s = launch_x(p, xj);
    if (s != SPADJ_OK) return s;
    YJobs yj{};
    for (int q = 0; q < 3; ++q) yj.j[q] = yfwd(ym(q), 1.0 / My, zm(q));
    yj.n = 3;
    if ((s = launch_y(p, yj)) != SPADJ_OK) return s;
    ZJobs zj = zjobs(0);
    for (int q = 0; q < 3; ++q) zj.j[q] = zfld(zm(q), gzF.as<double>(), 0, fld(f, nfield, q));
    zj.n = 3;
    return launch_z(p, zj);
  }

  spadj_status evalF(Problem* p, const double2* x, double2* f, DevBuf& G) {
    spadj_status s = c2g6(p, x, G);
    if (s != SPADJ_OK) return s;
    if (!nonlinear) {
      SPADJ_CUDA_TRY(p, cudaMemsetAsync(f, 0, sizeof(double2) * ns, p->stream));
      return SPADJ_OK;
    }
    return g2c3(p, f, G.as<double>(), nullptr);
  }

  spadj_status evalJvp(Problem* p, DevBuf& G, const double2* dx, double2* df) {
    if (!nonlinear) {
      SPADJ_CUDA_TRY(p, cudaMemsetAsync(df, 0, sizeof(double2) * ns, p->stream));
      return SPADJ_OK;
    }
    spadj_status s = c2g6(p, dx, dGf);
    if (s != SPADJ_OK) return s;
    return g2c3(p, df, G.as<double>(), dGf.as<double>());
  }

  // out = sum_a beta_a add_a + (dF/dx)(x)^H (sum_t alpha_t fb_t), grid fields of x in G
  spadj_status evalVjp(Problem* p, DevBuf& G, int nfb, const double2* const* fb, const double* alpha, int nadd,
                       const double2* const* add, const double* beta, double2* out) {
    spadj_status s;
    if (!nonlinear) {
      if (nadd == 0) {
        SPADJ_CUDA_TRY(p, cudaMemsetAsync(out, 0, sizeof(double2) * ns, p->stream));
        return SPADJ_OK;
      }
      axpy_kernel<<<256, 256, 0, p->stream>>>(out, add[0], beta[0], nadd > 1 ? add[1] : nullptr,
                                              nadd > 1 ? beta[1] : 0.0, nadd > 2 ? add[2] : nullptr,
                                              nadd > 2 ? beta[2] : 0.0, ns);
      return check_launch(p, "couette axpy");
    }
    // T^dagger: Gz^T in z, zero-pad + inverse FFT / My in y, c2r with weights 1/Mx, 1/(2Mx) in x
    ZJobs zj = zjobs(1);
    for (int q = 0; q < 3; ++q) {
      ZJob j = zexp(nullptr, gzTE.as<double>(), 0, zm(q));
      for (int t = 0; t < nfb; ++t) {
        j.xin[t] = fb[t] + (size_t)q * nfield; j.xalpha[t] = alpha[t]; j.xmult[t] = 0; j.xterm[t] = 0;
      }
      j.nx = nfb;
      zj.j[q] = j;
    }
    zj.n = 3;
    if ((s = launch_z(p, zj)) != SPADJ_OK) return s;
    YJobs yj{};
    for (int q = 0; q < 3; ++q) {
      yj.j[q] = yinv(ym(q), 1.0 / My);
      yadd(yj.j[q], zm(q), 1.0, 0);
    }
    yj.n = 3;
    if ((s = launch_y(p, yj)) != SPADJ_OK) return s;
    XJobs xj{};
    for (int q = 0; q < 3; ++q) xj.j[q] = xc2r(ym(q), 1.0 / Mx, 0.5 / Mx, grid(Fg, q));
    xj.n = 3;
    if ((s = launch_x(p, xj)) != SPADJ_OK) return s;
    cudaEvent_t tp = p->tic();
    const int pg = (int)std::min<size_t>((npts + 255) / 256, 4096);
    SPADJ_CUDA_TRY(p, launch_kernel(p->pdl, cou_prod_vjp_kernel, dim3(pg), dim3(256), 0, p->stream,
                                    (const double*)G.as<double>(), (const double*)Fg.as<double>(), Gb.as<double>(), npts));
    p->toc(tp, KC_POINTWISE, 18.0 * npts);
    if ((s = check_launch(p, "couette prod vjp")) != SPADJ_OK) return s;
    // (T^-1)^dagger: r2c with factor 2 on kx >= 1, forward FFT in y (truncated), then z folds
    XJobs xb{};
    for (int q = 0; q < 6; ++q) xb.j[q] = xr2c(grid(Gb, q), 1.0, 2.0, ym(q));
    xb.n = 6;
    if ((s = launch_x(p, xb)) != SPADJ_OK) return s;
    YJobs yb{};
    for (int q = 0; q < 6; ++q) yb.j[q] = yfwd(ym(q), 1.0, zm(q));
    yb.n = 6;
    if ((s = launch_y(p, yb)) != SPADJ_OK) return s;
    // ubar = Cz^T (c_u + i ky c_oz) + (Cz Dz)^T c_oy
    // vbar = Cz^T (c_v - i kx c_oz) - (Cz Dz)^T c_ox
    // wbar = Cz^T (c_w - i ky c_ox + i kx c_oy)
    ZJobs zf = zjobs(0);
    for (int q = 0; q < 3; ++q) {
      ZJob j = zfld(zm(q), czTF.as<double>(), 0, fld(out, nfield, q));
      if (q == 0) {
        j.xin[0] = zm(5); j.xalpha[0] = 1.0; j.xmult[0] = 2; j.xterm[0] = 0; j.nx = 1;
        j.in[1] = zm(4); j.mat[1] = cdzTF.as<double>(); j.alpha[1] = 1.0; j.deriv[1] = 1; j.nterm = 2;
      } else if (q == 1) {
        j.xin[0] = zm(5); j.xalpha[0] = -1.0; j.xmult[0] = 1; j.xterm[0] = 0; j.nx = 1;
        j.in[1] = zm(3); j.mat[1] = cdzTF.as<double>(); j.alpha[1] = -1.0; j.deriv[1] = 1; j.nterm = 2;
      } else {
        j.xin[0] = zm(3); j.xalpha[0] = -1.0; j.xmult[0] = 2; j.xterm[0] = 0;
        j.xin[1] = zm(4); j.xalpha[1] = 1.0; j.xmult[1] = 1; j.xterm[1] = 0;
        j.nx = 2;
      }
      for (int a = 0; a < nadd; ++a) { j.add[a] = add[a] + (size_t)q * nfield; j.beta[a] = beta[a]; }
      j.nadd = nadd;
      zf.j[q] = j;
    }
    zf.n = 3;
    return launch_z(p, zf);
  }

  // The dense step operators Phi of both scheme orders (couette_setup.h, build_phi).
  spadj_status ensure_dense(Problem* p) {
    if (dense_ok) return SPADJ_OK;
    std::string err;
    for (int ord = 1; ord <= order; ++ord) {
      std::vector<double> f, a;
      if (!couhost::build_phi(ops, Kx, Ny, Lx, Ly, nu, ord == 1 ? 1.0 / dt : 1.5 / dt, f, a, &err, base))
        return p->fail(SPADJ_ERR_INVALID, err);
      DevBuf& F = ord == 1 ? phi1F : phi2F;
      DevBuf& A = ord == 1 ? phi1A : phi2A;
      SPADJ_CUDA_TRY(p, F.ensure(sizeof(double) * f.size()));
      SPADJ_CUDA_TRY(p, A.ensure(sizeof(double) * a.size()));
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(F.ptr, f.data(), sizeof(double) * f.size(), cudaMemcpyHostToDevice, p->stream));
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(A.ptr, a.data(), sizeof(double) * a.size(), cudaMemcpyHostToDevice, p->stream));
      SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    }
    dense_ok = true;
    return SPADJ_OK;
  }

  // The banded factors of both scheme orders and directions (couette_setup.h, build_band).
  // Widths beyond the kernel's rounds (kl > 32, ku > 64) leave the banded form off: the dense
  // operators serve the solves instead.
  spadj_status ensure_band(Problem* p) {
    if (band_ok) return SPADJ_OK;
    if (band_too_wide) return ensure_dense(p);
    std::string err;
    for (int ord = 1; ord <= order; ++ord)
      for (int dir = 0; dir < 2; ++dir) {
        couhost::BandFactors F;
        if (!couhost::build_band(ops, Kx, Ny, Lx, Ly, nu, ord == 1 ? 1.0 / dt : 1.5 / dt, base, dir == 1, F, &err))
          return p->fail(SPADJ_ERR_INVALID, err);
        if (F.kl > 32 || F.ku > 64) {  // remembered: the factorisation is not repeated on every solve
          band_too_wide = true;
          return ensure_dense(p);
        }
        BandDev& B = band[ord - 1][dir];
        B.kl = F.kl;
        B.ku = F.ku;
        B.nv = F.nv;
        auto put = [&](DevBuf& b, const void* h, size_t bytes) -> cudaError_t {
          cudaError_t e = b.ensure(bytes);
          if (e != cudaSuccess) return e;
          return cudaMemcpyAsync(b.ptr, h, bytes, cudaMemcpyHostToDevice, p->stream);
        };
        SPADJ_CUDA_TRY(p, put(B.L, F.L.data(), sizeof(double) * F.L.size()));
        SPADJ_CUDA_TRY(p, put(B.U, F.U.data(), sizeof(double) * F.U.size()));
        SPADJ_CUDA_TRY(p, put(B.dinv, F.dinv.data(), sizeof(double) * F.dinv.size()));
        SPADJ_CUDA_TRY(p, put(B.piv, F.piv.data(), F.piv.size()));
        SPADJ_CUDA_TRY(p, put(B.ssb, F.ssb.data(), sizeof(double) * F.ssb.size()));
        SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
      }
    band_ok = true;
    return SPADJ_OK;
  }

  bool use_band(const Problem* p) const { return p->cou_band < 0 ? band_auto : p->cou_band != 0; }

  // x = P Phi v (transpose = 0) or v = Phi^H P x (transpose = 1), v = sum_t a_t in_t;
  // scheme order 1 or 2 selects the SBDF1 or SBDF2 operator.  The banded factors serve the
  // solve unless option 12 selects the dense Phi (or the band is too wide for the kernel).
  spadj_status solve(Problem* p, int transpose, int ord, int nin, const double2* const* in, const double* a,
                     double2* out) {
    if (use_band(p)) {
      spadj_status s = ensure_band(p);
      if (s != SPADJ_OK) return s;
      if (band_ok) return solve_band(p, transpose, ord, nin, in, a, out);
    }
    spadj_status s = ensure_dense(p);
    if (s != SPADJ_OK) return s;
    return solve_with(p, transpose, (ord == 1 ? phi1F : phi2F).as<double2>(), (ord == 1 ? phi1A : phi2A).as<double2>(),
                      1, nin, in, a, out);
  }

  template <int RL, int RU>
  cudaError_t launch_band(Problem* p, size_t smem, const CouBandArgs& S) {
    return launch_kernel(p->pdl, cou_band_kernel<RL, RU>, dim3(Kx * (Ny / 2 + 1)), dim3(32), smem, p->stream, S);
  }
  spadj_status solve_band(Problem* p, int transpose, int ord, int nin, const double2* const* in, const double* a,
                          double2* out) {
    const BandDev& B = band[ord - 1][transpose ? 1 : 0];
    CouBandArgs S{};
    for (int t = 0; t < nin; ++t) { S.in[t] = in[t]; S.a[t] = a[t]; }
    S.nin = nin; S.out = out; S.transpose = transpose;
    S.L = B.L.as<double2>(); S.U = B.U.as<double2>(); S.dinv = B.dinv.as<double2>();
    S.piv = B.piv.as<unsigned char>(); S.ssb = B.ssb.as<double>();
    S.kl = B.kl; S.ku = B.ku; S.nv = B.nv;
    S.Kx = Kx; S.Ny = Ny; S.N = N;
    const size_t smem = sizeof(double2) * (2 * (size_t)B.nv + 6 * (size_t)N);
    const int rl = (2 * B.kl + 31) / 32, ru = (2 * B.ku + 31) / 32;
    cudaEvent_t t = p->tic();
    cudaError_t e;
    if (rl <= 1) {
      e = ru <= 1 ? launch_band<1, 1>(p, smem, S) : ru == 2 ? launch_band<1, 2>(p, smem, S)
        : ru == 3 ? launch_band<1, 3>(p, smem, S) : launch_band<1, 4>(p, smem, S);
    } else {
      e = ru <= 1 ? launch_band<2, 1>(p, smem, S) : ru == 2 ? launch_band<2, 2>(p, smem, S)
        : ru == 3 ? launch_band<2, 3>(p, smem, S) : launch_band<2, 4>(p, smem, S);
    }
    SPADJ_CUDA_TRY(p, e);
    // complex multiply-adds of the two sweeps and the scaling, per right-hand side
    p->toc(t, KC_SOLVE, (8.0 * (B.kl + B.ku) + 6.0) * B.nv * (double)Kx * (Ny - 1));
    return check_launch(p, "couette banded solve");
  }
  spadj_status solve_with(Problem* p, int transpose, const double2* phiF_, const double2* phiA_, int project, int nin,
                          const double2* const* in, const double* a, double2* out) {
    CouSolveArgs S{};
    for (int t = 0; t < nin; ++t) { S.in[t] = in[t]; S.a[t] = a[t]; }
    S.nin = nin; S.out = out; S.transpose = transpose;
    S.phiF = phiF_;
    S.phiA = phiA_;
    S.project = project;
    S.Kx = Kx; S.Ny = Ny; S.N = N;
    const int H = 3 * N;
    const int threads = ((H + 31) / 32) * 32;
    cudaEvent_t t = p->tic();
    SPADJ_CUDA_TRY(p, launch_kernel(p->pdl, cou_solve_kernel, dim3(Kx, Ny / 2 + 1), dim3(threads),
                                    sizeof(double2) * 2 * H, p->stream, S));
    p->toc(t, KC_SOLVE, 8.0 * H * H * (double)Kx * (Ny - 1));
    return check_launch(p, "couette solve");
  }

  // scheme coefficients of step n (eq. imex): a[0..2], c[0..2] and the operator order
  int step_order(int n) const { return (n <= 1 || order == 1) ? 1 : 2; }
  void coeffs(int n, double* a, double* c) const {
    if (step_order(n) == 1) {
      a[0] = 1.0 / dt; a[1] = -1.0 / dt; a[2] = 0.0;
      c[0] = 0.0; c[1] = 1.0; c[2] = 0.0;
    } else {
      a[0] = 1.5 / dt; a[1] = -2.0 / dt; a[2] = 0.5 / dt;
      c[0] = 0.0; c[1] = 2.0; c[2] = -1.0;
    }
  }

  // x_n = P Phi_n (c1 f_{n-1} + c2 f_{n-2} - a1 x_{n-1} - a2 x_{n-2})
  spadj_status step(Problem* p, int n, const double2* xc, const double2* xp_, const double2* fc, const double2* fp,
                    double2* xn) {
    double a[3], c[3];
    coeffs(n, a, c);
    if (step_order(n) == 1) {
      const double2* in[2] = {fc, xc};
      double w[2] = {c[1], -a[1]};
      return solve(p, 0, 1, 2, in, w, xn);
    }
    const double2* in[4] = {fc, fp, xc, xp_};
    double w[4] = {c[1], c[2], -a[1], -a[2]};
    return solve(p, 0, 2, 4, in, w, xn);
  }

  // Forward sweep state: X ring (cur, prev, next) and F ring (cur, prev).
  struct Ring {
    int xc = 0, xp = 1, xn = 2, fc = 0, fp = 1;
    void advance() {
      const int t = xp;
      xp = xc;
      xc = xn;
      xn = t;
      std::swap(fc, fp);
    }
  };

  spadj_status advance(Problem* p, Ring& r, int n) {
    spadj_status s = evalF(p, st(Xr, r.xc), st(Fr, r.fc), Gf);
    if (s != SPADJ_OK) return s;
    if ((s = step(p, n, st(Xr, r.xc), st(Xr, r.xp), st(Fr, r.fc), st(Fr, r.fp), st(Xr, r.xn))) != SPADJ_OK) return s;
    r.advance();
    return SPADJ_OK;
  }

  spadj_status forward(Problem* p, int n_steps, const double* x0, double* x_out, double* traj) override {
    if (n_steps < 0) return p->fail(SPADJ_ERR_INVALID, "forward: n_steps < 0");
    const size_t sb = sizeof(double2) * ns;
    Ring r;
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(Xr, r.xc), x0, sb, cudaMemcpyDeviceToDevice, p->stream));
    if (traj) SPADJ_CUDA_TRY(p, cudaMemcpyAsync(traj, x0, sb, cudaMemcpyDeviceToDevice, p->stream));
    for (int n = 1; n <= n_steps; ++n) {
      spadj_status s = advance(p, r, n);
      if (s != SPADJ_OK) return s;
      if (traj)
        SPADJ_CUDA_TRY(p, cudaMemcpyAsync(reinterpret_cast<double2*>(traj) + (size_t)n * ns, st(Xr, r.xc), sb,
                                          cudaMemcpyDeviceToDevice, p->stream));
    }
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(x_out, st(Xr, r.xc), sb, cudaMemcpyDeviceToDevice, p->stream));
    return SPADJ_OK;
  }

  spadj_status tangent(Problem* p, int n_steps, const double* x0, const double* dx0, double* dx_out) override {
    if (n_steps < 0) return p->fail(SPADJ_ERR_INVALID, "tangent: n_steps < 0");
    const size_t sb = sizeof(double2) * ns;
    SPADJ_CUDA_TRY(p, dXr.ensure(3 * sb));
    SPADJ_CUDA_TRY(p, dFr.ensure(2 * sb));
    Ring r;
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(Xr, r.xc), x0, sb, cudaMemcpyDeviceToDevice, p->stream));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(dXr, r.xc), dx0, sb, cudaMemcpyDeviceToDevice, p->stream));
    for (int n = 1; n <= n_steps; ++n) {
      spadj_status s;
      if ((s = evalF(p, st(Xr, r.xc), st(Fr, r.fc), Gf)) != SPADJ_OK) return s;
      if ((s = evalJvp(p, Gf, st(dXr, r.xc), st(dFr, r.fc))) != SPADJ_OK) return s;
      if ((s = step(p, n, st(Xr, r.xc), st(Xr, r.xp), st(Fr, r.fc), st(Fr, r.fp), st(Xr, r.xn))) != SPADJ_OK)
        return s;
      if ((s = step(p, n, st(dXr, r.xc), st(dXr, r.xp), st(dFr, r.fc), st(dFr, r.fp), st(dXr, r.xn))) != SPADJ_OK)
        return s;
      r.advance();
    }
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(dx_out, st(dXr, r.xc), sb, cudaMemcpyDeviceToDevice, p->stream));
    return SPADJ_OK;
  }

  // ---- reverse sweep -------------------------------------------------------------------------
  double2* W(int n) { return st(Wr, n % 3); }

  // xbar_k from W_{k+1}, W_{k+2} (when k + i <= n_steps), the primal x_k and src (nullable);
  // then W_k = Phi_k^H P xbar_k for k >= 1.
  spadj_status reverse_index(Problem* p, int k, int n_steps, const double2* xk, const double2* src, double2* xb) {
    spadj_status s;
    const double2* fb[2];
    double al[2];
    int nfb = 0;
    const double2* ad[3];
    double be[3];
    int nad = 0;
    double a[3], c[3];
    if (k + 1 <= n_steps) {
      coeffs(k + 1, a, c);
      fb[nfb] = W(k + 1); al[nfb++] = c[1];
      ad[nad] = W(k + 1); be[nad++] = -a[1];
    }
    if (k + 2 <= n_steps && step_order(k + 2) == 2) {
      coeffs(k + 2, a, c);
      fb[nfb] = W(k + 2); al[nfb++] = c[2];
      ad[nad] = W(k + 2); be[nad++] = -a[2];
    }
    if (src) { ad[nad] = src; be[nad++] = 1.0; }
    if (nonlinear && nfb > 0) {
      if ((s = c2g6(p, xk, Gf)) != SPADJ_OK) return s;
      if ((s = evalVjp(p, Gf, nfb, fb, al, nad, ad, be, xb)) != SPADJ_OK) return s;
    } else if (nad > 0) {
      axpy_kernel<<<256, 256, 0, p->stream>>>(xb, ad[0], be[0], nad > 1 ? ad[1] : nullptr, nad > 1 ? be[1] : 0.0,
                                              nad > 2 ? ad[2] : nullptr, nad > 2 ? be[2] : 0.0, ns);
      if ((s = check_launch(p, "couette axpy")) != SPADJ_OK) return s;
    } else {
      SPADJ_CUDA_TRY(p, cudaMemsetAsync(xb, 0, sizeof(double2) * ns, p->stream));
    }
    if (k >= 1) {
      const double2* in[1] = {xb};
      double w[1] = {1.0};
      return solve(p, 1, step_order(k), 1, in, w, W(k));
    }
    return SPADJ_OK;
  }

  spadj_status energy(Problem* p, const double2* x, double* e_out, const double* scale, double2* seed) {
    cudaEvent_t t = p->tic();
    cou_energy_kernel<<<P, 128, 0, p->stream>>>(x, gmat.as<double>(), Kx, Ny, N, partial.as<double>(), scale, seed);
    p->toc(t, KC_OBJECTIVE, 4.0 * (double)P * 3 * N * N);  // real N x N matrix times complex vector: 2 FMA per entry
    spadj_status s = check_launch(p, "couette energy");
    if (s != SPADJ_OK) return s;
    sum_kernel<<<1, 128, 0, p->stream>>>(partial.as<double>(), P, e_out);
    return check_launch(p, "couette sum");
  }

  // J and dJ/dx at the final state x (and, for the gain, the X_0 source into src0 when x0src)
  spadj_status objective_at(Problem* p, int kind, const double2* x0, const double2* x, double* J_dev, double2* seed,
                            bool x0src) {
    spadj_status s;
    if (kind == SPADJ_OBJ_ENERGY) {
      if ((s = energy(p, x, J_dev, one.as<double>(), seed)) != SPADJ_OK) return s;
      return SPADJ_OK;
    }
    if (kind != SPADJ_OBJ_GAIN) return p->fail(SPADJ_ERR_UNSUPPORTED, "couette: objective must be ENERGY or GAIN");
    if (!x0) return p->fail(SPADJ_ERR_INVALID, "couette: the GAIN objective needs X_0 (obj_data)");
    double* e = edev.as<double>();
    double* sc = sdev.as<double>();
    if ((s = energy(p, x0, e, nullptr, nullptr)) != SPADJ_OK) return s;
    if ((s = energy(p, x, e + 1, nullptr, nullptr)) != SPADJ_OK) return s;
    gain_kernel<<<1, 1, 0, p->stream>>>(e, J_dev, sc);
    if ((s = check_launch(p, "couette gain")) != SPADJ_OK) return s;
    if ((s = energy(p, x, e + 1, sc, seed)) != SPADJ_OK) return s;  // dJ/dX_N = grad E(X_N) / E_0
    if (x0src && (s = energy(p, x0, e, sc + 1, src0.as<double2>())) != SPADJ_OK) return s;  // -E_N/E_0^2 grad E(X_0)
    return SPADJ_OK;
  }

  spadj_status objective(Problem* p, int kind, const double* obj_data, const double* x, double* J_dev,
                         double* sd) override {
    return objective_at(p, kind, reinterpret_cast<const double2*>(obj_data), reinterpret_cast<const double2*>(x),
                        J_dev, reinterpret_cast<double2*>(sd), false);
  }

  int last_recompute = 0;

  // Checkpointed reverse sweep over augmented states (x_n, x_{n-1}, f_{n-1}) (the restart data
  // of the two-step scheme).  objective_kind >= 0: seeds from the objective; < 0: caller seeds.
  spadj_status reverse(Problem* p, const double* x0, int n_steps, int ckpt_slots, int objective_kind,
                       const std::vector<int>& seed_at, const double* seeds, double* J_host, double* grad) {
    if (n_steps < 1) return p->fail(SPADJ_ERR_INVALID, "gradient: n_steps < 1");
    if (objective_kind >= 0 && objective_kind != SPADJ_OBJ_ENERGY && objective_kind != SPADJ_OBJ_GAIN &&
        objective_kind != SPADJ_OBJ_ENERGY_INTEGRAL)
      return p->fail(SPADJ_ERR_UNSUPPORTED, "couette: objective must be ENERGY, GAIN or ENERGY_INTEGRAL");
    const bool integral = objective_kind == SPADJ_OBJ_ENERGY_INTEGRAL;
    if (integral) {
      // dI/dt = E(X) added to the equation set (M = 1, L = 0 for I): the scalar adjoint of the
      // I-equation, a_0^m Y_m = [m == N] - sum_i a_i^{m+i} Y_{m+i}, gives the weight
      // s_n = sum_i c_i^{n+i} Y_{n+i} with which grad E(X_n) enters the state adjoint, and
      // I_N = sum_n s_n E(X_n)
      std::vector<double> Y((size_t)n_steps + 3, 0.0), sw((size_t)n_steps, 0.0);
      double a[3], c[3];
      for (int m = n_steps; m >= 1; --m) {
        double r = (m == n_steps) ? 1.0 : 0.0;
        for (int i = 1; i <= 2; ++i) {
          if (m + i > n_steps) continue;
          coeffs(m + i, a, c);
          r -= a[i] * Y[m + i];
        }
        coeffs(m, a, c);
        Y[m] = r / a[0];
      }
      for (int n = 0; n < n_steps; ++n)
        for (int i = 1; i <= 2; ++i) {
          if (n + i > n_steps) continue;
          coeffs(n + i, a, c);
          sw[n] += c[i] * Y[n + i];
        }
      SPADJ_CUDA_TRY(p, wts.ensure(sizeof(double) * (size_t)n_steps));
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(wts.ptr, sw.data(), sizeof(double) * n_steps, cudaMemcpyHostToDevice, p->stream));
      SPADJ_CUDA_TRY(p, cudaMemsetAsync(Jdev.ptr, 0, sizeof(double), p->stream));
      SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));  // the host weights go out of scope
    }
    const int S = (ckpt_slots <= 0 || ckpt_slots > n_steps + 1) ? n_steps + 1 : ckpt_slots;
    const size_t sb = sizeof(double2) * ns;
    SPADJ_CUDA_TRY(p, slots.ensure(3 * sb * (size_t)S));
    CkptPlanner planner;
    const int H = std::min(p->host_slots, n_steps);
    std::vector<CkptOp> ops = H > 0 ? planner.plan2(n_steps, S, H) : planner.plan(n_steps, S);
    if (H > 0) SPADJ_CUDA_TRY(p, hslots.ensure(3 * sb * (size_t)H));
    const double2* x0c = reinterpret_cast<const double2*>(x0);
    Ring r;
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(Xr, r.xc), x0, sb, cudaMemcpyDeviceToDevice, p->stream));
    int cur_step = 0, recompute = 0;
    bool have_seed = false;
    // device slots 0..S-1, host slots S..S+H-1; each holds (x_n, x_{n-1}, f_{n-1})
    auto slot = [&](int sl, int part) {
      return sl < S ? slots.as<char>() + ((size_t)sl * 3 + part) * sb
                    : hslots.as<char>() + ((size_t)(sl - S) * 3 + part) * sb;
    };
    auto seed_ptr = [&](int n) -> const double2* {
      if (objective_kind >= 0 || n < 0 || n >= (int)seed_at.size() || seed_at[n] < 0) return nullptr;
      return reinterpret_cast<const double2*>(seeds) + (size_t)seed_at[n] * ns;
    };
    for (const CkptOp& op : ops) {
      spadj_status s = SPADJ_OK;
      switch (op.type) {
        case CK_STORE: {
          const cudaMemcpyKind k = op.slot < S ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
          SPADJ_CUDA_TRY(p, cudaMemcpyAsync(slot(op.slot, 0), st(Xr, r.xc), sb, k, p->stream));
          SPADJ_CUDA_TRY(p, cudaMemcpyAsync(slot(op.slot, 1), st(Xr, r.xp), sb, k, p->stream));
          SPADJ_CUDA_TRY(p, cudaMemcpyAsync(slot(op.slot, 2), st(Fr, r.fp), sb, k, p->stream));
          break;
        }
        case CK_RESTORE:
          if (cur_step != op.a) {
            const cudaMemcpyKind k = op.slot < S ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
            SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(Xr, r.xc), slot(op.slot, 0), sb, k, p->stream));
            SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(Xr, r.xp), slot(op.slot, 1), sb, k, p->stream));
            SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(Fr, r.fp), slot(op.slot, 2), sb, k, p->stream));
            cur_step = op.a;
          }
          break;
        case CK_ADVANCE:
          for (int n = op.a + 1; n <= op.b; ++n) {
            if ((s = advance(p, r, n)) != SPADJ_OK) return s;
            ++recompute;
          }
          cur_step = op.b;
          break;
        case CK_OBJECTIVE: {
          double2* xb = xbar.as<double2>();
          if (integral) {
            SPADJ_CUDA_TRY(p, cudaMemsetAsync(xb, 0, sb, p->stream));  // J = I_N has no X_N term
          } else if (objective_kind >= 0) {
            if ((s = objective_at(p, objective_kind, x0c, st(Xr, r.xc), Jdev.as<double>(), xb,
                                  objective_kind == SPADJ_OBJ_GAIN)) != SPADJ_OK)
              return s;
          } else if (const double2* sp = seed_ptr(n_steps)) {
            SPADJ_CUDA_TRY(p, cudaMemcpyAsync(xb, sp, sb, cudaMemcpyDeviceToDevice, p->stream));
          } else {
            SPADJ_CUDA_TRY(p, cudaMemsetAsync(xb, 0, sb, p->stream));
          }
          const double2* in[1] = {xb};
          double w[1] = {1.0};
          if ((s = solve(p, 1, step_order(n_steps), 1, in, w, W(n_steps))) != SPADJ_OK) return s;
          have_seed = true;
          break;
        }
        case CK_ADJOINT: {
          if (!have_seed)
            return p->fail(SPADJ_ERR_INVALID, "gradient: schedule reached an adjoint step before the objective");
          const int k = op.a;
          const double2* src = seed_ptr(k);
          if (objective_kind == SPADJ_OBJ_GAIN && k == 0) src = src0.as<double2>();
          if (integral) {  // s_k grad E(X_k) into src0, and J += s_k E(X_k)
            const double* wk = wts.as<double>() + k;
            if ((s = energy(p, st(Xr, r.xc), edev.as<double>(), wk, src0.as<double2>())) != SPADJ_OK) return s;
            integral_accum_kernel<<<1, 1, 0, p->stream>>>(edev.as<double>(), wk, Jdev.as<double>());
            if ((s = check_launch(p, "couette integral")) != SPADJ_OK) return s;
            src = src0.as<double2>();
          }
          if ((s = reverse_index(p, k, n_steps, st(Xr, r.xc), src, xbar.as<double2>())) != SPADJ_OK) return s;
          break;
        }
        default:
          break;
      }
    }
    last_recompute = recompute;
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(grad, xbar.ptr, sb, cudaMemcpyDeviceToDevice, p->stream));
    if (J_host && objective_kind >= 0) {
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(J_host, Jdev.ptr, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
      SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
      if (!std::isfinite(J_host[0])) return p->fail(SPADJ_ERR_NONFINITE, "couette: objective is not finite");
    }
    return SPADJ_OK;
  }

  spadj_status adjoint(Problem* p, int n_steps, const double* traj, const double* y_final, double* grad,
                       double* grad_p) override {
    if (n_steps < 1) return p->fail(SPADJ_ERR_INVALID, "adjoint: n_steps < 1");
    if (grad_p) return p->fail(SPADJ_ERR_UNSUPPORTED, "couette: the problem has no parameters (grad_p must be NULL)");
    const size_t sb = sizeof(double2) * ns;
    const double2* tr = reinterpret_cast<const double2*>(traj);
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(xbar.ptr, y_final, sb, cudaMemcpyDeviceToDevice, p->stream));
    {
      const double2* in[1] = {xbar.as<double2>()};
      double w[1] = {1.0};
      spadj_status s = solve(p, 1, step_order(n_steps), 1, in, w, W(n_steps));
      if (s != SPADJ_OK) return s;
    }
    for (int k = n_steps - 1; k >= 0; --k) {
      spadj_status s = reverse_index(p, k, n_steps, tr + (size_t)k * ns, nullptr, xbar.as<double2>());
      if (s != SPADJ_OK) return s;
    }
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(grad, xbar.ptr, sb, cudaMemcpyDeviceToDevice, p->stream));
    return SPADJ_OK;
  }

  spadj_status gradient(Problem* p, const double* x0, int n_steps, int objective_kind, const double* obj_data,
                        int ckpt_slots, double* J_host, double* grad, double* grad_p) override {
    (void)obj_data;
    if (grad_p) return p->fail(SPADJ_ERR_UNSUPPORTED, "couette: the problem has no parameters (grad_p must be NULL)");
    return reverse(p, x0, n_steps, ckpt_slots, objective_kind, {}, nullptr, J_host, grad);
  }

  spadj_status vjp(Problem* p, const double* x0, int n_steps, int ckpt_slots, const std::vector<int>& seed_at,
                   const double* seeds, double* grad) override {
    return reverse(p, x0, n_steps, ckpt_slots, -1, seed_at, seeds, nullptr, grad);
  }

  // ---- one step at a time ----------------------------------------------------------------------
  // Restart state of step n (X_n -> X_{n+1}): [x_n, x_{n-1}, f_{n-1}] (SBDF2; [x_n] for SBDF1), the
  // augmented state the checkpoint slots hold.  Adjoint state: [Y_n, Y_{n+1}] (SBDF2; [Y_n] for
  // SBDF1), the adjoint variables of eq. IMEX_adjoint in prognostic form (Y_m = Phi_m^H P xbar_m),
  // the same vectors the reverse sweep keeps in its W ring.
  int step_blocks(int which) const override { return which == 0 ? 2 * order - 1 : order; }

  spadj_status step_forward(Problem* p, int n, const double* s_n, double* s_np1) override {
    if (n < 0) return p->fail(SPADJ_ERR_INVALID, "step: n < 0");
    const size_t sb = sizeof(double2) * ns;
    const double2* in = reinterpret_cast<const double2*>(s_n);
    double2* out = reinterpret_cast<double2*>(s_np1);
    Ring r;
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(Xr, r.xc), in, sb, cudaMemcpyDeviceToDevice, p->stream));
    if (order == 2) {
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(Xr, r.xp), in + ns, sb, cudaMemcpyDeviceToDevice, p->stream));
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(Fr, r.fp), in + 2 * ns, sb, cudaMemcpyDeviceToDevice, p->stream));
    }
    spadj_status s = advance(p, r, n + 1);
    if (s != SPADJ_OK) return s;
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(out, st(Xr, r.xc), sb, cudaMemcpyDeviceToDevice, p->stream));
    if (order == 2) {
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(out + ns, st(Xr, r.xp), sb, cudaMemcpyDeviceToDevice, p->stream));
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(out + 2 * ns, st(Fr, r.fp), sb, cudaMemcpyDeviceToDevice, p->stream));
    }
    return SPADJ_OK;
  }

  spadj_status step_tangent(Problem* p, int n, const double* s_n, const double* ds_n, double* ds_np1) override {
    if (n < 0) return p->fail(SPADJ_ERR_INVALID, "step: n < 0");
    const size_t sb = sizeof(double2) * ns;
    SPADJ_CUDA_TRY(p, dXr.ensure(3 * sb));
    SPADJ_CUDA_TRY(p, dFr.ensure(2 * sb));
    const double2* in = reinterpret_cast<const double2*>(s_n);
    const double2* din = reinterpret_cast<const double2*>(ds_n);
    double2* dout = reinterpret_cast<double2*>(ds_np1);
    Ring r;
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(Xr, r.xc), in, sb, cudaMemcpyDeviceToDevice, p->stream));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(dXr, r.xc), din, sb, cudaMemcpyDeviceToDevice, p->stream));
    if (order == 2) {
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(Xr, r.xp), in + ns, sb, cudaMemcpyDeviceToDevice, p->stream));
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(Fr, r.fp), in + 2 * ns, sb, cudaMemcpyDeviceToDevice, p->stream));
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(dXr, r.xp), din + ns, sb, cudaMemcpyDeviceToDevice, p->stream));
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(dFr, r.fp), din + 2 * ns, sb, cudaMemcpyDeviceToDevice, p->stream));
    }
    spadj_status s;
    if ((s = evalF(p, st(Xr, r.xc), st(Fr, r.fc), Gf)) != SPADJ_OK) return s;
    if ((s = evalJvp(p, Gf, st(dXr, r.xc), st(dFr, r.fc))) != SPADJ_OK) return s;
    if ((s = step(p, n + 1, st(dXr, r.xc), st(dXr, r.xp), st(dFr, r.fc), st(dFr, r.fp), st(dXr, r.xn))) != SPADJ_OK)
      return s;
    r.advance();
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(dout, st(dXr, r.xc), sb, cudaMemcpyDeviceToDevice, p->stream));
    if (order == 2) {
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(dout + ns, st(dXr, r.xp), sb, cudaMemcpyDeviceToDevice, p->stream));
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(dout + 2 * ns, st(dFr, r.fp), sb, cudaMemcpyDeviceToDevice, p->stream));
    }
    return SPADJ_OK;
  }

  // eq. IMEX_adjoint at index n: xbar_n = sum_i (c_i^{n+i} J(X_n) - a_i^{n+i} M)^dagger Y_{n+i} + src,
  // then Y_n = Phi_n^H P xbar_n (n >= 1); at n = 0 the first block of y_n is xbar_0 = dJ/dX_0.
  // y_np1 = NULL stands for zero adjoint variables (the seed step at n = N with src = dJ/dX_N).
  spadj_status step_adjoint(Problem* p, int n, const double* x_n, const double* y_np1, const double* src, double* y_n,
                            double* gp_accum) override {
    if (gp_accum) return p->fail(SPADJ_ERR_INVALID, "couette: the problem has no parameters (gp_accum must be NULL)");
    if (n < 0) return p->fail(SPADJ_ERR_INVALID, "step: n < 0");
    const size_t sb = sizeof(double2) * ns;
    const double2* yin = reinterpret_cast<const double2*>(y_np1);
    double2* yout = reinterpret_cast<double2*>(y_n);
    double2* xb = xbar.as<double2>();
    spadj_status s;
    if (!yin) {
      if (src) SPADJ_CUDA_TRY(p, cudaMemcpyAsync(xb, src, sb, cudaMemcpyDeviceToDevice, p->stream));
      else SPADJ_CUDA_TRY(p, cudaMemsetAsync(xb, 0, sb, p->stream));
      if (order == 2) SPADJ_CUDA_TRY(p, cudaMemsetAsync(W(n + 1), 0, sb, p->stream));
    } else {
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(W(n + 1), yin, sb, cudaMemcpyDeviceToDevice, p->stream));
      if (order == 2) SPADJ_CUDA_TRY(p, cudaMemcpyAsync(W(n + 2), yin + ns, sb, cudaMemcpyDeviceToDevice, p->stream));
      // every later step exists: the adjoint variables past the horizon are the caller's zeros
      if ((s = reverse_index(p, n, 1 << 29, reinterpret_cast<const double2*>(x_n),
                             reinterpret_cast<const double2*>(src), xb)) != SPADJ_OK)
        return s;
    }
    if (n >= 1 && !yin) {
      const double2* in[1] = {xb};
      double w[1] = {1.0};
      if ((s = solve(p, 1, step_order(n), 1, in, w, W(n))) != SPADJ_OK) return s;
    }
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(yout, n >= 1 ? W(n) : xb, sb, cudaMemcpyDeviceToDevice, p->stream));
    if (order == 2) SPADJ_CUDA_TRY(p, cudaMemcpyAsync(yout + ns, W(n + 1), sb, cudaMemcpyDeviceToDevice, p->stream));
    return SPADJ_OK;
  }

  // ---- Hessian-vector product ----------------------------------------------------------------
  // hv = (d^2 J / dX_0^2) v for J = E(X_N): forward sweep with its tangent along v (both
  // trajectories stored), then the adjoint recurrence and its tangent together.  F = u x omega
  // is quadratic, so the tangent of (dF/dx)(x_k)^H w along dx_k is (dF/dx)(dx_k)^H w: the VJP
  // evaluated with the grid fields of dx_k.  The objective's Hessian is grad E (linear).
  spadj_status hvp(Problem* p, const double* x0, const double* v, int n_steps, double* hv) {
    if (n_steps < 1) return p->fail(SPADJ_ERR_INVALID, "hvp: n_steps < 1");
    const size_t sb = sizeof(double2) * ns;
    SPADJ_CUDA_TRY(p, htraj.ensure(sb * ((size_t)n_steps + 1)));
    SPADJ_CUDA_TRY(p, hdtraj.ensure(sb * ((size_t)n_steps + 1)));
    SPADJ_CUDA_TRY(p, dWr.ensure(3 * sb));
    SPADJ_CUDA_TRY(p, dxbar.ensure(sb));
    SPADJ_CUDA_TRY(p, htmp.ensure(sb));
    SPADJ_CUDA_TRY(p, dXr.ensure(3 * sb));
    SPADJ_CUDA_TRY(p, dFr.ensure(2 * sb));
    double2* X = htraj.as<double2>();
    double2* dX = hdtraj.as<double2>();
    auto xs = [&](double2* base, int n) { return base + (size_t)n * ns; };
    // forward and tangent, stored
    Ring r;
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(Xr, r.xc), x0, sb, cudaMemcpyDeviceToDevice, p->stream));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(st(dXr, r.xc), v, sb, cudaMemcpyDeviceToDevice, p->stream));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(xs(X, 0), x0, sb, cudaMemcpyDeviceToDevice, p->stream));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(xs(dX, 0), v, sb, cudaMemcpyDeviceToDevice, p->stream));
    spadj_status s;
    for (int n = 1; n <= n_steps; ++n) {
      if ((s = evalF(p, st(Xr, r.xc), st(Fr, r.fc), Gf)) != SPADJ_OK) return s;
      if ((s = evalJvp(p, Gf, st(dXr, r.xc), st(dFr, r.fc))) != SPADJ_OK) return s;
      if ((s = step(p, n, st(Xr, r.xc), st(Xr, r.xp), st(Fr, r.fc), st(Fr, r.fp), st(Xr, r.xn))) != SPADJ_OK) return s;
      if ((s = step(p, n, st(dXr, r.xc), st(dXr, r.xp), st(dFr, r.fc), st(dFr, r.fp), st(dXr, r.xn))) != SPADJ_OK)
        return s;
      r.advance();
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(xs(X, n), st(Xr, r.xc), sb, cudaMemcpyDeviceToDevice, p->stream));
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(xs(dX, n), st(dXr, r.xc), sb, cudaMemcpyDeviceToDevice, p->stream));
    }
    // seeds at X_N: grad E(X_N) and its tangent grad E(dX_N)
    double2* xb = xbar.as<double2>();
    double2* dxb = dxbar.as<double2>();
    auto dW = [&](int n) { return st(dWr, n % 3); };
    if ((s = energy(p, xs(X, n_steps), edev.as<double>(), one.as<double>(), xb)) != SPADJ_OK) return s;
    if ((s = energy(p, xs(dX, n_steps), edev.as<double>() + 1, one.as<double>(), dxb)) != SPADJ_OK) return s;
    { const double2* in[1] = {xb}; double w1[1] = {1.0};
      if ((s = solve(p, 1, step_order(n_steps), 1, in, w1, W(n_steps))) != SPADJ_OK) return s; }
    { const double2* in[1] = {dxb}; double w1[1] = {1.0};
      if ((s = solve(p, 1, step_order(n_steps), 1, in, w1, dW(n_steps))) != SPADJ_OK) return s; }
    for (int k = n_steps - 1; k >= 0; --k) {
      const double2* fb[2];
      const double2* dfb[2];
      double al[2];
      int nfb = 0;
      const double2* ad[2];
      const double2* dad[2];
      double be[2];
      int nad = 0;
      double a[3], c[3];
      if (k + 1 <= n_steps) {
        coeffs(k + 1, a, c);
        fb[nfb] = W(k + 1); dfb[nfb] = dW(k + 1); al[nfb++] = c[1];
        ad[nad] = W(k + 1); dad[nad] = dW(k + 1); be[nad++] = -a[1];
      }
      if (k + 2 <= n_steps && step_order(k + 2) == 2) {
        coeffs(k + 2, a, c);
        fb[nfb] = W(k + 2); dfb[nfb] = dW(k + 2); al[nfb++] = c[2];
        ad[nad] = W(k + 2); dad[nad] = dW(k + 2); be[nad++] = -a[2];
      }
      if (nonlinear) {
        if ((s = c2g6(p, xs(X, k), Gf)) != SPADJ_OK) return s;
        if ((s = evalVjp(p, Gf, nfb, fb, al, nad, ad, be, xb)) != SPADJ_OK) return s;
        if ((s = evalVjp(p, Gf, nfb, dfb, al, nad, dad, be, htmp.as<double2>())) != SPADJ_OK) return s;
        if ((s = c2g6(p, xs(dX, k), dGf)) != SPADJ_OK) return s;
        const double2* ad1[1] = {htmp.as<double2>()};
        double be1[1] = {1.0};
        if ((s = evalVjp(p, dGf, nfb, fb, al, 1, ad1, be1, dxb)) != SPADJ_OK) return s;
      } else {
        axpy_kernel<<<256, 256, 0, p->stream>>>(xb, ad[0], be[0], nad > 1 ? ad[1] : nullptr, nad > 1 ? be[1] : 0.0,
                                                nullptr, 0.0, ns);
        axpy_kernel<<<256, 256, 0, p->stream>>>(dxb, dad[0], be[0], nad > 1 ? dad[1] : nullptr, nad > 1 ? be[1] : 0.0,
                                                nullptr, 0.0, ns);
        if ((s = check_launch(p, "couette axpy")) != SPADJ_OK) return s;
      }
      if (k >= 1) {
        { const double2* in[1] = {xb}; double w1[1] = {1.0};
          if ((s = solve(p, 1, step_order(k), 1, in, w1, W(k))) != SPADJ_OK) return s; }
        { const double2* in[1] = {dxb}; double w1[1] = {1.0};
          if ((s = solve(p, 1, step_order(k), 1, in, w1, dW(k))) != SPADJ_OK) return s; }
      }
    }
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(hv, dxb, sb, cudaMemcpyDeviceToDevice, p->stream));
    return SPADJ_OK;
  }

  // ---- resolvent gains -----------------------------------------------------------------------
  // Leading gain per (kx, ky) pencil of the resolvent R(omega) = [(i omega M + L)^-1]_prog S1S0
  // in the energy norm ||c||^2 = c^H G c per field: power iteration on the generalised problem
  // R^H G R f = sigma^2 G f, all pencils at once.  f (state layout) holds the initial forcing on
  // entry and the leading forcing (unit energy per pencil) on exit; gains[Ny][Kx] the gains.
  spadj_status resolvent(Problem* p, double omega, int n_iter, double* f_io, double* gains) {
    if (n_iter < 1) return p->fail(SPADJ_ERR_INVALID, "resolvent: n_iter < 1");
    if (!res_built || omega != res_omega) {
      std::vector<double> rf, ra;
      std::string err;
      if (!couhost::build_phi(ops, Kx, Ny, Lx, Ly, nu, std::complex<double>(0.0, omega), rf, ra, &err, base))
        return p->fail(SPADJ_ERR_INVALID, err);
      SPADJ_CUDA_TRY(p, phiRF.ensure(sizeof(double) * rf.size()));
      SPADJ_CUDA_TRY(p, phiRA.ensure(sizeof(double) * ra.size()));
      SPADJ_CUDA_TRY(p, cudaMemcpy(phiRF.ptr, rf.data(), sizeof(double) * rf.size(), cudaMemcpyHostToDevice));
      SPADJ_CUDA_TRY(p, cudaMemcpy(phiRA.ptr, ra.data(), sizeof(double) * ra.size(), cudaMemcpyHostToDevice));
      res_built = true;
      res_omega = omega;
    }
    if (!ginv.ptr) {  // G^-1 by Gauss-Jordan elimination with partial pivoting (G is SPD, N x N)
      std::vector<double> A(ops.G), I((size_t)N * N, 0.0);
      for (int i = 0; i < N; ++i) I[(size_t)i * N + i] = 1.0;
      for (int k = 0; k < N; ++k) {
        int piv = k;
        for (int i = k + 1; i < N; ++i)
          if (std::fabs(A[(size_t)i * N + k]) > std::fabs(A[(size_t)piv * N + k])) piv = i;
        for (int j = 0; j < N; ++j) {
          std::swap(A[(size_t)k * N + j], A[(size_t)piv * N + j]);
          std::swap(I[(size_t)k * N + j], I[(size_t)piv * N + j]);
        }
        const double d = A[(size_t)k * N + k];
        for (int j = 0; j < N; ++j) { A[(size_t)k * N + j] /= d; I[(size_t)k * N + j] /= d; }
        for (int i = 0; i < N; ++i) {
          if (i == k) continue;
          const double l = A[(size_t)i * N + k];
          if (l == 0.0) continue;
          for (int j = 0; j < N; ++j) { A[(size_t)i * N + j] -= l * A[(size_t)k * N + j]; I[(size_t)i * N + j] -= l * I[(size_t)k * N + j]; }
        }
      }
      std::vector<double> IT(I.size());  // stored transposed for cou_gram_kernel (G itself is symmetric)
      for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) IT[(size_t)j * N + i] = I[(size_t)i * N + j];
      SPADJ_CUDA_TRY(p, ginv.ensure(sizeof(double) * IT.size()));
      SPADJ_CUDA_TRY(p, cudaMemcpy(ginv.ptr, IT.data(), sizeof(double) * IT.size(), cudaMemcpyHostToDevice));
    }
    SPADJ_CUDA_TRY(p, nrm.ensure(sizeof(double) * P));
    SPADJ_CUDA_TRY(p, g2.ensure(sizeof(double) * P));
    double2* f = reinterpret_cast<double2*>(f_io);
    double2* y = st(Wr, 0);
    double2* z = st(Wr, 1);
    double2* t = st(Wr, 2);
    spadj_status s;
    auto gram = [&](const double2* in, const DevBuf& mat, double2* out, double* nr) -> spadj_status {
      cudaEvent_t ev = p->tic();
      cou_gram_kernel<<<P, 128, 0, p->stream>>>(in, mat.as<double>(), Kx, Ny, N, out, nr);
      p->toc(ev, KC_GRAM, 4.0 * (double)P * 3 * N * N);  // real N x N matrix times complex vector: 2 FMA per entry
      return check_launch(p, "couette gram");
    };
    auto normalise = [&](double* gout) -> spadj_status {
      if ((s = gram(f, gmat, t, nrm.as<double>())) != SPADJ_OK) return s;
      cou_pencil_scale_kernel<<<P, 128, 0, p->stream>>>(f, nrm.as<double>(), Kx, Ny, N, g2.as<double>(), gout);
      return check_launch(p, "couette scale");
    };
    if ((s = normalise(nullptr)) != SPADJ_OK) return s;
    const double one_[1] = {1.0};
    for (int it = 0; it < n_iter; ++it) {
      { const double2* in[1] = {f};
        if ((s = solve_with(p, 0, phiRF.as<double2>(), phiRA.as<double2>(), 0, 1, in, one_, y)) != SPADJ_OK) return s; }
      if ((s = gram(y, gmat, z, g2.as<double>())) != SPADJ_OK) return s;  // ||R f||_G^2 with ||f||_G = 1
      { const double2* in[1] = {z};
        if ((s = solve_with(p, 1, phiRF.as<double2>(), phiRA.as<double2>(), 0, 1, in, one_, t)) != SPADJ_OK) return s; }
      if ((s = gram(t, ginv, f, nullptr)) != SPADJ_OK) return s;
      if ((s = normalise(it + 1 == n_iter ? gains : nullptr)) != SPADJ_OK) return s;
    }
    return SPADJ_OK;
  }

  // ---- single operations ---------------------------------------------------------------------
  spadj_status transform(Problem* p, int kind, const double* in, double* out) override {
    const double2* ci = reinterpret_cast<const double2*>(in);
    double2* co = reinterpret_cast<double2*>(out);
    spadj_status s;
    if (kind == 0 || kind == 3) {
      ZJobs zj = zjobs(1);
      zj.j[0] = zexp(ci, kind == 0 ? czE.as<double>() : gzTE.as<double>(), 0, zm(0));
      zj.n = 1;
      if ((s = launch_z(p, zj)) != SPADJ_OK) return s;
      YJobs yj{};
      yj.j[0] = yinv(ym(0), kind == 0 ? 1.0 : 1.0 / My);
      yadd(yj.j[0], zm(0), 1.0, 0);
      yj.n = 1;
      if ((s = launch_y(p, yj)) != SPADJ_OK) return s;
      XJobs xj{};
      xj.j[0] = kind == 0 ? xc2r(ym(0), 1.0, 1.0, out) : xc2r(ym(0), 1.0 / Mx, 0.5 / Mx, out);
      xj.n = 1;
      return launch_x(p, xj);
    }
    if (kind == 1 || kind == 2) {
      XJobs xj{};
      xj.j[0] = kind == 1 ? xr2c(in, 1.0 / Mx, 1.0 / Mx, ym(0)) : xr2c(in, 1.0, 2.0, ym(0));
      xj.n = 1;
      if ((s = launch_x(p, xj)) != SPADJ_OK) return s;
      YJobs yj{};
      yj.j[0] = yfwd(ym(0), kind == 1 ? 1.0 / My : 1.0, zm(0));
      yj.n = 1;
      if ((s = launch_y(p, yj)) != SPADJ_OK) return s;
      ZJobs zj = zjobs(0);
      zj.j[0] = zfld(zm(0), kind == 1 ? gzF.as<double>() : czTF.as<double>(), 0, co);
      zj.n = 1;
      return launch_z(p, zj);
    }
    return p->fail(SPADJ_ERR_INVALID, "transform: kind must be 0..3");
  }

  spadj_status eval_F(Problem* p, int mode, const double* x, const double* dx, double* out) override {
    const double2* xc = reinterpret_cast<const double2*>(x);
    const double2* dc = reinterpret_cast<const double2*>(dx);
    double2* oc = reinterpret_cast<double2*>(out);
    spadj_status s;
    if (mode == 0) return evalF(p, xc, oc, Gf);
    if ((s = c2g6(p, xc, Gf)) != SPADJ_OK) return s;
    if (mode == 1) return evalJvp(p, Gf, dc, oc);
    const double2* fb[1] = {dc};
    double al[1] = {1.0};
    return evalVjp(p, Gf, 1, fb, al, 0, nullptr, nullptr, oc);
  }

  spadj_status pencil_solve(Problem* p, int transpose, const double* v, double* x) {
    const double2* in[1] = {reinterpret_cast<const double2*>(v)};
    double a[1] = {1.0};
    return solve(p, transpose, order, 1, in, a, reinterpret_cast<double2*>(x));
  }

  ~Couette() override {
    for (auto& o2 : band)
      for (BandDev& B : o2)
        for (DevBuf* b : {&B.L, &B.U, &B.dinv, &B.piv, &B.ssb}) b->release();
    for (DevBuf* b : {&wmx, &w2y, &czE, &cdzE, &gzF, &gzTE, &czTF, &cdzTF, &gmat, &phi1F, &phi1A, &phi2F, &phi2A, &one,
                      &Zm, &Ym, &Gf, &dGf, &Gb, &Fg, &Xr, &Fr, &dXr, &dFr, &Wr, &xbar, &src0, &partial, &edev, &sdev,
                      &Jdev, &slots, &wts, &phiRF, &phiRA, &ginv, &nrm, &g2, &htraj, &hdtraj, &dWr, &dxbar, &htmp})
      b->release();
    hslots.release();
  }
};

}  // namespace

EqImpl* make_couette(Problem* p, spadj_status* st) {
  Couette* c = new Couette();
  *st = c->init(p);
  if (*st != SPADJ_OK) {
    delete c;
    return nullptr;
  }
  return c;
}

spadj_status cou_hvp(EqImpl* impl, Problem* p, const double* x0, const double* v, int n_steps, double* hv) {
  Couette* c = dynamic_cast<Couette*>(impl);
  if (!c) return p->fail(SPADJ_ERR_UNSUPPORTED, "hvp: only defined for the plane-Couette problem");
  return c->hvp(p, x0, v, n_steps, hv);
}

spadj_status cou_resolvent(EqImpl* impl, Problem* p, double omega, int n_iter, double* f, double* gains) {
  Couette* c = dynamic_cast<Couette*>(impl);
  if (!c) return p->fail(SPADJ_ERR_UNSUPPORTED, "resolvent: only defined for the plane-Couette problem");
  return c->resolvent(p, omega, n_iter, f, gains);
}

spadj_status cou_pencil_solve(EqImpl* impl, Problem* p, int transpose, const double* v, double* x) {
  Couette* c = dynamic_cast<Couette*>(impl);
  if (!c) return p->fail(SPADJ_ERR_UNSUPPORTED, "solve: not a plane-Couette problem");
  return c->pencil_solve(p, transpose, v, x);
}

}  // namespace spadj
