// 2D Rayleigh-Benard convection: RK222 IMEX forward step, tangent step and exact discrete
// adjoint step on the GPU, with binomial checkpointing for the gradient.
//
// Per RK222 step (ARS(2,2,2), Supplementary A.4, both stages share M + dt*gamma*L):
//   f0 = F(x0);  v1 = x0 + dt A10 f0;                      x1 = Phi v1
//   f1 = F(x1);  v2 = (1-c) x0 + dt(A20 - c A10) f0 + dt A21 f1 + c x1;   x2 = Phi v2
// where every quantity is in Chebyshev-T space, Phi is the per-pencil prognostic stage
// solution operator (rb_setup.cpp) and c = H21/gamma: the stage-2 term -dt H21 L X1 equals
// -(H21/gamma)(R1 - M X1) because X1 solves (M + dt gamma L) X1 = R1, and R1 - M X1 =
// S1S0 (v1 - x1).  The adjoint step is the exact reverse of this sequence (it equals the
// paper's RK IMEX adjoint recurrence; the parity tests check it against the oracle's
// implementation of that recurrence), the tangent its forward derivative.
// F is evaluated pseudospectrally: z transforms (Chebyshev matrices with reflection
// folding), x FFTs, grid products, back to T space (Sparse spectral methods section).
#include <cmath>
#include <functional>
#include <memory>
#include <string>
#include <mutex>
#include <vector>

#include "problem.h"
#include "rb_kernels.cuh"
#include "rb_setup.h"
#include "revolve.h"

namespace spadj {
namespace {

using namespace rbk;

struct RB : EqImpl {
  // sizes and parameters
  int Nx = 0, Kx = 0, N = 0, Mx = 0, Mz = 0, L = 0;
  double Lx = 4.0, nu = 0, kappa = 0, dt = 0, Ra = 0, Pr = 1;
  double A10, A20, A21, H21, gam, cc;
  // generic Runge-Kutta IMEX path (ARS(4,4,3)): S implicit stages, tableaux tA (explicit) and
  // tH (implicit, diagonal gam, zero first column)
  bool generic = false;
  int S = 2;
  double tA[5][5] = {}, tH[5][5] = {};
  int nonlinear = 1;
  size_t ns = 0;    // complex entries of one state [3][Kx][N]
  size_t nmix = 0;  // complex entries of one mixed array [Mz][Kx]
  size_t npts = 0;  // grid points Mz*Mx
  XParams xp{};
  // device constants
  DevBuf wm, czE, cdzE, gzF, gzTE, czTF, cdzTF, gmat;
  // Stage solution operators and the step graphs that use them, one set per step size: the
  // base dt of the descriptor, plus one per distinct size of a step-size schedule
  // (spadj_set_dt_schedule), factorised when first needed and kept (Methods: the LU
  // decompositions are reused unless the timestep changes).
  struct OpSet {
    double dt = 0.0;
    DevBuf phi, phiT;
    cudaGraphExec_t gFwd[2] = {nullptr, nullptr};
    cudaGraphExec_t gFwdB[2] = {nullptr, nullptr};  // lane 1 forward step graphs
    cudaGraphExec_t gAdj[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    cudaGraphExec_t gStage[2] = {nullptr, nullptr};                           // lane 2 stage-1 graphs
    cudaGraphExec_t gAdjS[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // lane 0 staged adjoint
  };
  std::vector<std::unique_ptr<OpSet>> opsets;
  OpSet* ops_cur = nullptr;
  double dt_base = 0.0;
  std::vector<double> sched;  // per-step sizes (empty: dt_base for every step)
  rbhost::Operators hops;     // host operators for later factorisations
  // device work buffers
  DevBuf dG, Gb, Fg, df0, df1, dx1, vb2, vb1, xb1, tmpx, tmpy, ybar, ybar2, cur, nxt, curB, nxtB, partial, Jdev,
      seedbuf, slots, traj_tmp;
  DevBuf errbuf;   // set by a fused column stage whose bounded wait for its operator block ran out
  HostBuf hslots;  // host tier of the two-level checkpoint schedule
  // Buffers of one forward step.  Lane 0 runs the forward sweep and the adjoint steps, lane 1
  // the recomputation of checkpointed segments, concurrently on its own stream; in the reverse
  // sweep of the fused scheme lane 2 computes the stage-1 grid fields of the next adjoint steps
  // into ws[2], ws[3] (alternating by step parity).
  struct WS {
    DevBuf Z, Y, G0, G1, f0, f1, x1;
    DevBuf rx[4], rv[4], rf[4];  // generic scheme: stage values x_i, pre-solve vectors v_i, F(x_{i-1})
  };
  // generic scheme, lane 0: tangent stages and adjoint cotangents
  DevBuf tdx[4], tdv[4], tdf[4], axb[4], avb[4], afb[4], aacc, atmp, axs;
  WS ws[4];
  WS* w = &ws[0];
  size_t zsmem = 0, xsmem = 0, ssmem = 0, csmem = 0, ctsmem = 0;
  bool fused = false;  // fused column stage (rb_colstep_kernel) usable for these sizes
  int xnb = 1;         // x-FFT launch variant, xvar(rows per CTA, threads) (tuned at creation)
  // internal streams (joined to the caller's stream by events) and captured step graphs
  cudaStream_t gs = nullptr, gs2 = nullptr, gsB = nullptr, gsC = nullptr;
  cudaEvent_t evIn = nullptr, evOut = nullptr, evFork = nullptr, evJoin = nullptr;
  cudaEvent_t evReady = nullptr, evFree = nullptr, evBdone = nullptr;  // lane handoffs
  cudaEvent_t evAdj[2] = {nullptr, nullptr}, evCopied[2] = {nullptr, nullptr};
  cudaEvent_t evStaged[2] = {nullptr, nullptr}, evCdone = nullptr;  // lane 2 handoffs
  double2* Sb[2] = {nullptr, nullptr};  // state ping-pong buffers
  double2* SbB[2] = {nullptr, nullptr};  // lane 1 state ping-pong buffers
  double2* Yb[2] = {nullptr, nullptr};  // cotangent ping-pong buffers

  size_t state_len(int which) const override {
    if (which == 0) return 2 * ns;
    if (which == 1) return npts;
    if (which == 3) return (size_t)2 * Kx * N;
    return 0;
  }

  double2* st(DevBuf& b, int f = 0) { return b.as<double2>() + (size_t)f * Kx * N; }
  double2* mix(DevBuf& b, int i) { return b.as<double2>() + (size_t)i * nmix; }
  double* grid(DevBuf& b, int i) { return b.as<double>() + (size_t)i * npts; }

  spadj_status init(Problem* p) {
    const spadj_desc& d = p->desc;
    Nx = d.n[0];
    N = d.n[1];
    if (Nx < 4 || Nx % 4 != 0 || N < 8 || N % 4 != 0)
      return p->fail(SPADJ_ERR_INVALID, "rb: n[0] must be a multiple of 4 (>= 4) and n[1] a multiple of 4 (>= 8)");
    if (d.scheme != SPADJ_RK222 && d.scheme != SPADJ_RK443)
      return p->fail(SPADJ_ERR_UNSUPPORTED, "rb: scheme must be RK222 or RK443");
    generic = d.scheme == SPADJ_RK443;
    if (d.batch != 1) return p->fail(SPADJ_ERR_UNSUPPORTED, "rb: batch must be 1 (one problem per handle)");
    Kx = Nx / 2;
    Mx = 3 * Nx / 2;
    Mz = 3 * N / 2;
    L = Mx / 2;
    if (Mz % 2 != 0) return p->fail(SPADJ_ERR_INVALID, "rb: 3*n[1]/2 must be even");
    Lx = d.length[0] > 0 ? d.length[0] : 4.0;
    Ra = d.params[0];
    Pr = d.params[1] > 0 ? d.params[1] : 1.0;
    if (!(Ra > 0)) return p->fail(SPADJ_ERR_INVALID, "rb: params[0] (Rayleigh number) must be > 0");
    nu = std::pow(Ra / Pr, -0.5);
    kappa = std::pow(Ra * Pr, -0.5);
    dt = d.dt;
    nonlinear = d.nonlinear;
    gam = 1.0 - 1.0 / std::sqrt(2.0);
    const double del = 1.0 - 1.0 / (2.0 * gam);
    A10 = gam; A20 = del; A21 = 1.0 - del; H21 = 1.0 - gam;
    cc = H21 / gam;
    if (generic) {  // ARS(4,4,3), Ascher, Ruuth & Spiteri (1997)
      S = 4;
      gam = 0.5;
      const double a[5][5] = {{0, 0, 0, 0, 0},
                              {1.0 / 2.0, 0, 0, 0, 0},
                              {11.0 / 18.0, 1.0 / 18.0, 0, 0, 0},
                              {5.0 / 6.0, -5.0 / 6.0, 1.0 / 2.0, 0, 0},
                              {1.0 / 4.0, 7.0 / 4.0, 3.0 / 4.0, -7.0 / 4.0, 0}};
      const double h[5][5] = {{0, 0, 0, 0, 0},
                              {0, 1.0 / 2.0, 0, 0, 0},
                              {0, 1.0 / 6.0, 1.0 / 2.0, 0, 0},
                              {0, -1.0 / 2.0, 1.0 / 2.0, 1.0 / 2.0, 0},
                              {0, 3.0 / 2.0, -3.0 / 2.0, 1.0 / 2.0, 1.0 / 2.0}};
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) { tA[i][j] = a[i][j]; tH[i][j] = h[i][j]; }
    }
    ns = (size_t)3 * Kx * N;
    nmix = (size_t)Mz * Kx;
    npts = (size_t)Mz * Mx;
    xp.Kx = Kx; xp.Mx = Mx; xp.L = L; xp.kscale = 2.0 * M_PI / Lx;
    xp.plan = make_plan(L);
    if (xp.plan.nrad < 0) return p->fail(SPADJ_ERR_INVALID, "rb: 3*n[0]/4 must be of the form 2^a 3^b");

    // host operators and solution operators
    rbhost::Operators o = rbhost::build_operators(N, Mz);
    hops = o;
    dt_base = dt;
    // half matrices for the reflection-folded z transforms
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
    std::vector<double2> hwm(Mx);
    for (int m = 0; m < Mx; ++m) {
      const double th = -2.0 * M_PI * (double)m / (double)Mx;
      hwm[m] = make_double2(std::cos(th), std::sin(th));
    }
    {  // the butterflies' scaled-twiddle records follow the M-table in the same buffer
      const std::vector<double2> sct = scaled_twiddle_table(xp.plan);
      hwm.insert(hwm.end(), sct.begin(), sct.end());
    }
    auto up = [&](DevBuf& b, const void* h, size_t bytes) -> cudaError_t {
      cudaError_t e = b.ensure(bytes);
      if (e != cudaSuccess) return e;
      return cudaMemcpyAsync(b.ptr, h, bytes, cudaMemcpyHostToDevice, p->stream);
    };
    SPADJ_CUDA_TRY(p, up(wm, hwm.data(), sizeof(double2) * hwm.size()));
    SPADJ_CUDA_TRY(p, up(czE, hczE.data(), sizeof(double) * hczE.size()));
    SPADJ_CUDA_TRY(p, up(cdzE, hcdzE.data(), sizeof(double) * hcdzE.size()));
    SPADJ_CUDA_TRY(p, up(gzF, hgzF.data(), sizeof(double) * hgzF.size()));
    SPADJ_CUDA_TRY(p, up(gzTE, hgzTE.data(), sizeof(double) * hgzTE.size()));
    SPADJ_CUDA_TRY(p, up(czTF, hczTF.data(), sizeof(double) * hczTF.size()));
    SPADJ_CUDA_TRY(p, up(cdzTF, hcdzTF.data(), sizeof(double) * hcdzTF.size()));
    SPADJ_CUDA_TRY(p, up(gmat, o.G.data(), sizeof(double) * o.G.size()));
    SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    {
      spadj_status s = opset_for(p, dt_base, &ops_cur);
      if (s != SPADJ_OK) return s;
    }
    xp.WM = wm.as<double2>();
    bind_scaled_twiddles(xp.plan, xp.WM + Mx);
    // work buffers
    const size_t sb = sizeof(double2) * ns, mb = sizeof(double2) * nmix, gb = sizeof(double) * npts;
    for (WS& l : ws) {
      SPADJ_CUDA_TRY(p, l.Z.ensure(6 * mb));
      SPADJ_CUDA_TRY(p, l.Y.ensure(6 * mb));
      SPADJ_CUDA_TRY(p, l.G0.ensure(8 * gb));
      SPADJ_CUDA_TRY(p, l.G1.ensure(8 * gb));
      for (DevBuf* b : {&l.f0, &l.f1, &l.x1}) SPADJ_CUDA_TRY(p, b->ensure(sb));
    }
    if (generic) {
      for (WS* l : {&ws[0], &ws[1]})
        for (int i = 0; i < 4; ++i)
          for (DevBuf* b : {&l->rx[i], &l->rv[i], &l->rf[i]}) SPADJ_CUDA_TRY(p, b->ensure(sb));
      for (int i = 0; i < 4; ++i)
        for (DevBuf* b : {&tdx[i], &tdv[i], &tdf[i], &axb[i], &avb[i], &afb[i]}) SPADJ_CUDA_TRY(p, b->ensure(sb));
      for (DevBuf* b : {&aacc, &atmp, &axs}) SPADJ_CUDA_TRY(p, b->ensure(sb));
    }
    SPADJ_CUDA_TRY(p, dG.ensure(8 * gb));
    SPADJ_CUDA_TRY(p, Gb.ensure(8 * gb));
    SPADJ_CUDA_TRY(p, Fg.ensure(3 * gb));
    for (DevBuf* b : {&df0, &df1, &dx1, &vb2, &vb1, &xb1, &tmpx, &tmpy, &ybar, &ybar2, &cur, &nxt, &curB, &nxtB, &seedbuf})
      SPADJ_CUDA_TRY(p, b->ensure(sb));
    Sb[0] = cur.as<double2>(); Sb[1] = nxt.as<double2>();
    SbB[0] = curB.as<double2>(); SbB[1] = nxtB.as<double2>();
    Yb[0] = ybar.as<double2>(); Yb[1] = ybar2.as<double2>();
    SPADJ_CUDA_TRY(p, cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
    SPADJ_CUDA_TRY(p, cudaStreamCreateWithFlags(&gs2, cudaStreamNonBlocking));
    SPADJ_CUDA_TRY(p, cudaStreamCreateWithFlags(&gsB, cudaStreamNonBlocking));
    SPADJ_CUDA_TRY(p, cudaStreamCreateWithFlags(&gsC, cudaStreamNonBlocking));
    for (cudaEvent_t* e : {&evIn, &evOut, &evFork, &evJoin, &evReady, &evFree, &evBdone, &evAdj[0], &evAdj[1],
                           &evCopied[0], &evCopied[1], &evStaged[0], &evStaged[1], &evCdone})
      SPADJ_CUDA_TRY(p, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    SPADJ_CUDA_TRY(p, partial.ensure(sizeof(double) * Kx));
    SPADJ_CUDA_TRY(p, Jdev.ensure(sizeof(double)));
    SPADJ_CUDA_TRY(p, errbuf.ensure(sizeof(int)));
    SPADJ_CUDA_TRY(p, cudaMemsetAsync(errbuf.ptr, 0, sizeof(int), p->stream));
    zsmem = (size_t)2 * 2 * (size_t)std::max(N, Mz / 2) * kTM * sizeof(double2);
    xsmem = sizeof(double2) * (4 * L + Kx);
    const int H = 3 * (N / 2);
    ssmem = sizeof(double2) * (H + 4 * solve_rows(H)) + sizeof(double) * (size_t)H * solve_rows(H);
    csmem = colstep_smem(N, Mz);
    ctsmem = colstepT_smem(N, Mz);
    fused = nonlinear && !generic && std::max(csmem, ctsmem) <= 200 * 1024;
    if (fused) {
      SPADJ_CUDA_TRY(p, cudaFuncSetAttribute(rb_colstep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem));
      SPADJ_CUDA_TRY(p, cudaFuncSetAttribute(rb_colstepT_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ctsmem));
    }
    {  // x-FFT rows per CTA, timed on the eight inverse transforms of one F evaluation
      SPADJ_CUDA_TRY(p, cudaMemsetAsync(w->Z.ptr, 0, w->Z.bytes, p->stream));
      cudaError_t e = cudaSuccess;
      xnb = tune_xfft_rows(c2r_jobs(w->G0), xp, Mz, p->stream, p->x_rows, &e);
      SPADJ_CUDA_TRY(p, e);
    }
    if (ssmem > 48 * 1024)
      SPADJ_CUDA_TRY(p, cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssmem));
    return SPADJ_OK;
  }

  // Stage operator set for step size h: found among the factorised ones or built now (host
  // factorisation of M + h gam L per pencil, split into the two reflection-parity blocks, and
  // uploaded synchronously).
  spadj_status opset_for(Problem* p, double h, OpSet** out) {
    for (auto& os : opsets)
      if (os->dt == h) { *out = os.get(); return SPADJ_OK; }
    std::vector<double> ph;
    std::string err;
    if (!rbhost::build_phi(hops, Kx, Lx, nu, kappa, h * gam, ph, &err)) return p->fail(SPADJ_ERR_INVALID, err);
    const int Nh = N / 2, H = 3 * Nh, np = 3 * N;
    std::vector<double> pb((size_t)Kx * 2 * H * H), pbT((size_t)Kx * 2 * H * H);
    auto cls_idx = [&](int cls, int c) {  // class-local index -> global prognostic index
      const int f = c / Nh, hh = c % Nh;
      const int n = 2 * hh + ((f == 0) ? cls : 1 - cls);
      return f * N + n;
    };
    for (int m = 0; m < Kx; ++m)
      for (int cls = 0; cls < 2; ++cls)
        for (int r = 0; r < H; ++r)
          for (int c = 0; c < H; ++c) {
            const double v = ph[(size_t)m * np * np + (size_t)cls_idx(cls, r) * np + cls_idx(cls, c)];
            pb[(((size_t)m * 2 + cls) * H + r) * H + c] = v;   // [r][c]
            pbT[(((size_t)m * 2 + cls) * H + c) * H + r] = v;  // [c][r]
          }
    std::unique_ptr<OpSet> os(new OpSet());
    os->dt = h;
    SPADJ_CUDA_TRY(p, os->phi.ensure(sizeof(double) * pb.size()));
    SPADJ_CUDA_TRY(p, os->phiT.ensure(sizeof(double) * pbT.size()));
    SPADJ_CUDA_TRY(p, cudaMemcpy(os->phi.ptr, pb.data(), sizeof(double) * pb.size(), cudaMemcpyHostToDevice));
    SPADJ_CUDA_TRY(p, cudaMemcpy(os->phiT.ptr, pbT.data(), sizeof(double) * pbT.size(), cudaMemcpyHostToDevice));
    *out = os.get();
    opsets.push_back(std::move(os));
    return SPADJ_OK;
  }

  // Before a sweep of n_steps: every step size it uses has its operators (built here, never in
  // the middle of the sweep).
  spadj_status prepare_steps(Problem* p, int n_steps) {
    if (sched.empty()) return SPADJ_OK;
    if ((int)sched.size() < n_steps)
      return p->fail(SPADJ_ERR_INVALID, "rb: the step-size schedule is shorter than n_steps");
    OpSet* os = nullptr;
    for (int n = 0; n < n_steps; ++n) {
      spadj_status s = opset_for(p, sched[n], &os);
      if (s != SPADJ_OK) return s;
    }
    return SPADJ_OK;
  }

  // Make step n's size and operators current (host state read while its launches are built).
  // prepare_steps has built every set a sweep selects; a missing one is an internal error.
  spadj_status select_step(Problem* p, int n) {
    const double h = sched.empty() ? dt_base : sched[n];
    if (ops_cur && ops_cur->dt == h) { dt = h; return SPADJ_OK; }
    for (auto& os : opsets)
      if (os->dt == h) { ops_cur = os.get(); dt = h; return SPADJ_OK; }
    return p->fail(SPADJ_ERR_INVALID, "rb: no stage operators for this step size");
  }
  void select_base() {
    dt = dt_base;
    ops_cur = opsets.empty() ? nullptr : opsets[0].get();
  }

  spadj_status set_schedule(Problem* p, int n, const double* dts) {
    for (int i = 0; i < n; ++i)
      if (!(dts[i] > 0.0) || !std::isfinite(dts[i])) return p->fail(SPADJ_ERR_INVALID, "set_dt_schedule: step sizes must be > 0");
    sched.assign(dts, dts + n);
    select_base();
    return SPADJ_OK;
  }

  // ---- building blocks -----------------------------------------------------------------------
  // algorithmic FP64 flops: folded z transform = 4 flops per real-matrix x complex MAC over
  // Kx columns and N x Mz/2 entries per term; real FFT of Mx points = 2.5 Mx log2 Mx.
  double zflops(const ZJobs& js) const {
    double f = 0;
    for (int i = 0; i < js.n; ++i) f += 4.0 * Kx * N * (Mz / 2) * js.j[i].nterm;
    return f;
  }
  double xflops(const XJobs& js) const {
    double f = 0, one = 2.5 * Mx * std::log2((double)Mx) * Mz;
    for (int i = 0; i < js.n; ++i) f += one * (js.j[i].dir == 0 ? 1 : js.j[i].nr);
    return f;
  }
  spadj_status launch_z(Problem* p, ZJobs& js) {
    js.ncols = Kx;
    dim3 grid(Kx, js.n);
    const int threads = zmm_threads(js.expand, js.j[0].I);
    cudaEvent_t t = p->tic();
    SPADJ_CUDA_TRY(p, launch_kernel(p->pdl, zmm_kernel, grid, dim3(threads), zsmem, p->stream, js));
    p->toc(t, KC_ZTRANSFORM, zflops(js));
    return check_launch(p, "rb zmm");
  }
  spadj_status launch_x(Problem* p, XJobs& js) {
    cudaEvent_t t = p->tic();
    SPADJ_CUDA_TRY(p, launch_xfft(p->pdl, p->x_rows ? p->x_rows : xnb, js, xp, Mz, p->stream));
    p->toc(t, KC_XFFT, xflops(js));
    return check_launch(p, "rb xfft");
  }
  ZJob zexpand(const double2* in, const double* mat, int deriv, double2* out) {
    ZJob j{};
    j.in[0] = in; j.mat[0] = mat; j.alpha[0] = 1.0; j.deriv[0] = deriv; j.nterm = 1;
    j.out = out; j.I = Mz; j.K = N; j.ik = 1; j.im = N; j.oi = Kx; j.om = 1;
    return j;
  }
  ZJob zfold(const double2* in, const double* mat, int deriv, double2* out) {
    ZJob j{};
    j.in[0] = in; j.mat[0] = mat; j.alpha[0] = 1.0; j.deriv[0] = deriv; j.nterm = 1;
    j.out = out; j.I = N; j.K = Mz; j.ik = Kx; j.im = 1; j.oi = 1; j.om = N;
    return j;
  }
  XJob xc2r(const double2* in, int cmul, double w0, double w, double* out) {
    XJob j{};
    j.dir = 0; j.cin = in; j.cmul = cmul; j.w0 = w0; j.w = w; j.rout = out;
    return j;
  }
  XJob xr2c(const double* in0, int mul0, const double* in1, int mul1, double s0, double s, double2* out) {
    XJob j{};
    j.dir = 1; j.rin[0] = in0; j.rmul[0] = mul0; j.nr = 1;
    if (in1) { j.rin[1] = in1; j.rmul[1] = mul1; j.nr = 2; }
    j.s0 = s0; j.s = s; j.cout = out;
    return j;
  }

  // grid fields u, ux, uz, w, wx, wz, tx, tz of the state x (T space) into G
  spadj_status c2g_fields(Problem* p, const double2* x, DevBuf& G) {
    ZJobs zj{};
    zj.expand = 1;
    const double2* u = x;
    const double2* wf = x + (size_t)Kx * N;
    const double2* t = x + (size_t)2 * Kx * N;
    zj.j[0] = zexpand(u, czE.as<double>(), 0, mix(w->Z, 0));
    zj.j[1] = zexpand(u, cdzE.as<double>(), 1, mix(w->Z, 1));
    zj.j[2] = zexpand(wf, czE.as<double>(), 0, mix(w->Z, 2));
    zj.j[3] = zexpand(wf, cdzE.as<double>(), 1, mix(w->Z, 3));
    zj.j[4] = zexpand(t, czE.as<double>(), 0, mix(w->Z, 4));
    zj.j[5] = zexpand(t, cdzE.as<double>(), 1, mix(w->Z, 5));
    zj.n = 6;
    spadj_status s = launch_z(p, zj);
    if (s != SPADJ_OK) return s;
    return c2r_fields(p, G);
  }

  // x-inverse FFTs of the six mixed columns in Z into the eight grid fields of G
  spadj_status c2r_fields(Problem* p, DevBuf& G) {
    XJobs xj = c2r_jobs(G);
    return launch_x(p, xj);
  }
  XJobs c2r_jobs(DevBuf& G) {
    XJobs xj{};
    xj.j[0] = xc2r(mix(w->Z, 0), 0, 1.0, 1.0, grid(G, 0));
    xj.j[1] = xc2r(mix(w->Z, 0), 1, 1.0, 1.0, grid(G, 1));
    xj.j[2] = xc2r(mix(w->Z, 1), 0, 1.0, 1.0, grid(G, 2));
    xj.j[3] = xc2r(mix(w->Z, 2), 0, 1.0, 1.0, grid(G, 3));
    xj.j[4] = xc2r(mix(w->Z, 2), 1, 1.0, 1.0, grid(G, 4));
    xj.j[5] = xc2r(mix(w->Z, 3), 0, 1.0, 1.0, grid(G, 5));
    xj.j[6] = xc2r(mix(w->Z, 4), 1, 1.0, 1.0, grid(G, 6));
    xj.j[7] = xc2r(mix(w->Z, 5), 0, 1.0, 1.0, grid(G, 7));
    xj.n = 8;
    return xj;
  }

  // the three grid products of F (or of its JVP when dGp is non-null) -> T-space state f
  // (products formed inside the x-forward FFT; g2c: 1/Mx r2c, then Gz)
  spadj_status g2c3(Problem* p, double2* f, const double* Gp, const double* dGp) {
    spadj_status s = products_r2c(p, Gp, dGp);
    if (s != SPADJ_OK) return s;
    ZJobs zj{};
    zj.expand = 0;
    for (int q = 0; q < 3; ++q) zj.j[q] = zfold(mix(w->Y, q), gzF.as<double>(), 0, f + (size_t)q * Kx * N);
    zj.n = 3;
    return launch_z(p, zj);
  }

  // x-forward FFTs of the grid products F_q = -(u dx q + w dz q) (or their tangents when dGp is
  // non-null) into the mixed rows Y; slots 0 u, 1 ux, 2 uz, 3 w, 4 wx, 5 wz, 6 tx, 7 tz
  spadj_status products_r2c(Problem* p, const double* Gp, const double* dGp = nullptr) {
    XJobs xj{};
    static const int qx[3] = {1, 4, 6};
    for (int q = 0; q < 3; ++q) {
      xj.j[q] = xr2c(nullptr, 0, nullptr, 0, 1.0 / Mx, 1.0 / Mx, mix(w->Y, q));
      xj.j[q].nprod = 2;
      xj.j[q].pa[0] = 0; xj.j[q].pb[0] = qx[q]; xj.j[q].ps[0] = -1.0;
      xj.j[q].pa[1] = 3; xj.j[q].pb[1] = qx[q] + 1; xj.j[q].ps[1] = -1.0;
      xj.j[q].G = Gp;
      xj.j[q].dG = dGp;
      xj.j[q].npts = (int)npts;
      xj.j[q].nr = 1;
    }
    xj.n = 3;
    return launch_x(p, xj);
  }

  int prod_grid() const { return (int)std::min<size_t>((npts + 255) / 256, 1024); }

  // f = F(x) in T space; grid fields of x left in G
  spadj_status evalF(Problem* p, const double2* x, double2* f, DevBuf& G) {
    spadj_status s = c2g_fields(p, x, G);
    if (s != SPADJ_OK) return s;
    if (!nonlinear) {
      cudaMemsetAsync(f, 0, sizeof(double2) * ns, p->stream);
      return check_launch(p, "rb zero F");
    }
    return g2c3(p, f, G.as<double>(), nullptr);
  }

  // df = (dF/dx)(x) dx, with the grid fields of x already in G
  spadj_status evalJvp(Problem* p, DevBuf& G, const double2* dx, double2* df) {
    if (!nonlinear) {
      cudaMemsetAsync(df, 0, sizeof(double2) * ns, p->stream);
      return check_launch(p, "rb zero dF");
    }
    spadj_status s = c2g_fields(p, dx, dG);
    if (s != SPADJ_OK) return s;
    return g2c3(p, df, G.as<double>(), dG.as<double>());
  }

  // out = sum_a beta_a add_a + (dF/dx)(x)^dagger (sum_t alpha_t fb_t), grid fields of x in G.
  spadj_status evalVjp(Problem* p, DevBuf& G, int nfb, const double2* const* fb, const double* alpha, int nadd,
                       const double2* const* add, const double* beta, double2* out) {
    spadj_status s;
    if (nonlinear) {
      if ((s = vjp_expand(p, nfb, fb, alpha)) != SPADJ_OK) return s;
      if ((s = vjp_middle(p, G)) != SPADJ_OK) return s;
    }
    return vjp_fold(p, nadd, add, beta, out);
  }

  // T^dagger in z: Z_q = Gz^T (sum_t alpha_t fb_t) (one matrix pass on the combined column)
  spadj_status vjp_expand(Problem* p, int nfb, const double2* const* fb, const double* alpha) {
    ZJobs zj{};
    zj.expand = 1;
    for (int q = 0; q < 3; ++q) {
      ZJob j{};
      j.mat[0] = gzTE.as<double>(); j.alpha[0] = 1.0; j.deriv[0] = 0; j.nterm = 1;
      for (int t = 0; t < nfb; ++t) {
        j.xin[t] = fb[t] + (size_t)q * Kx * N; j.xalpha[t] = alpha[t]; j.xterm[t] = 0;
      }
      j.nx = nfb;
      j.out = mix(w->Z, q); j.I = Mz; j.K = N; j.ik = 1; j.im = N; j.oi = Kx; j.om = 1;
      zj.j[q] = j;
    }
    zj.n = 3;
    return launch_z(p, zj);
  }

  // from Z (T^dagger in z done): c2r with weights 1/Mx, 1/(2Mx), reverse of the grid products
  // with the fields G, then (T^-1)^dagger in x (r2c, factor 2 on k >= 1, -ik) into Y
  spadj_status vjp_middle(Problem* p, DevBuf& G) {
    spadj_status s;
    XJobs xj{};
    for (int q = 0; q < 3; ++q) xj.j[q] = xc2r(mix(w->Z, q), 0, 1.0 / Mx, 0.5 / Mx, grid(Fg, q));
    xj.n = 3;
    if ((s = launch_x(p, xj)) != SPADJ_OK) return s;
    cudaEvent_t tp = p->tic();
    SPADJ_CUDA_TRY(p, launch_kernel(p->pdl, prod_vjp_kernel, dim3(prod_grid()), dim3(256), 0, p->stream,
                                    (const double*)G.as<double>(), (const double*)Fg.as<double>(), Gb.as<double>(),
                                    (int)npts));
    p->toc(tp, KC_POINTWISE, 24.0 * npts);
    if ((s = check_launch(p, "rb prod vjp")) != SPADJ_OK) return s;
    XJobs xb{};
    xb.j[0] = xr2c(grid(Gb, 0), 0, grid(Gb, 1), 2, 1.0, 2.0, mix(w->Y, 0));  // a_u
    xb.j[1] = xr2c(grid(Gb, 2), 0, nullptr, 0, 1.0, 2.0, mix(w->Y, 1));      // b_u
    xb.j[2] = xr2c(grid(Gb, 3), 0, grid(Gb, 4), 2, 1.0, 2.0, mix(w->Y, 2));  // a_w
    xb.j[3] = xr2c(grid(Gb, 5), 0, nullptr, 0, 1.0, 2.0, mix(w->Y, 3));      // b_w
    xb.j[4] = xr2c(grid(Gb, 6), 2, nullptr, 0, 1.0, 2.0, mix(w->Y, 4));      // a_t
    xb.j[5] = xr2c(grid(Gb, 7), 0, nullptr, 0, 1.0, 2.0, mix(w->Y, 5));      // b_t
    xb.n = 6;
    return launch_x(p, xb);
  }

  // z part: out_q = Cz^T a_q + C'z^T b_q (+ addends)
  spadj_status vjp_fold(Problem* p, int nadd, const double2* const* add, const double* beta, double2* out) {
    ZJobs zf{};
    zf.expand = 0;
    for (int q = 0; q < 3; ++q) {
      ZJob j{};
      if (nonlinear) {
        j.in[0] = mix(w->Y, 2 * q); j.mat[0] = czTF.as<double>(); j.alpha[0] = 1.0; j.deriv[0] = 0;
        j.in[1] = mix(w->Y, 2 * q + 1); j.mat[1] = cdzTF.as<double>(); j.alpha[1] = 1.0; j.deriv[1] = 1;
        j.nterm = 2;
      } else {
        j.in[0] = mix(w->Y, 0); j.mat[0] = czTF.as<double>(); j.alpha[0] = 0.0; j.nterm = 1;
      }
      for (int a = 0; a < nadd; ++a) { j.add[a] = add[a] + (size_t)q * Kx * N; j.beta[a] = beta[a]; }
      j.nadd = nadd;
      j.out = out + (size_t)q * Kx * N; j.I = N; j.K = Mz; j.ik = Kx; j.im = 1; j.oi = 1; j.om = N;
      zf.j[q] = j;
    }
    zf.n = 3;
    if (!nonlinear) {
      // alpha = 0 term reads a mixed buffer that must be finite
      cudaMemsetAsync(w->Y.ptr, 0, sizeof(double2) * nmix, p->stream);
    }
    return launch_z(p, zf);
  }

  // fused adjoint column stage: xb = fold(Y) + sum_a beta_a add_a, vb = Phi^H xb (into vb),
  // Z = Gz^T (al0 c0 + al1 vb)
  spadj_status colstepT(Problem* p, int nadd, const double2* const* add, const double* beta, double2* vb,
                        const double2* c0, double al0, double al1) {
    ColStepTArgs S{};
    for (int e = 0; e < 6; ++e) S.yin[e] = mix(w->Y, e);
    S.czTF = czTF.as<double>();
    S.cdzTF = cdzTF.as<double>();
    for (int a = 0; a < nadd; ++a) { S.add[a] = add[a]; S.beta[a] = beta[a]; }
    S.nadd = nadd;
    S.phiA = ops_cur->phi.as<double>();
    S.v_out = vb;
    S.c0 = c0;
    S.al0 = al0;
    S.al1 = al1;
    S.gzTE = gzTE.as<double>();
    S.zout = w->Z.as<double2>();
    S.nmix = nmix;
    S.Kx = Kx; S.N = N; S.Mz = Mz;
    S.err = errbuf.as<int>();
    S.bulk = p->bulk_staging ? 1 : 0;
    const int H = 3 * N / 2;
    const double fl = (double)Kx * (3 * 2 * 4.0 * N * (Mz / 2) + 2 * 4.0 * H * H + 3 * 4.0 * N * (Mz / 2));
    cudaEvent_t t = p->tic();
    rb_colstepT_kernel<<<2 * Kx, 256, ctsmem, p->stream>>>(S);
    p->toc(t, KC_FUSED, fl);
    return check_launch(p, "rb colstepT");
  }

  // out = Phi (sum_t a_t in_t) (transpose 0) or Phi^H ... (transpose 1), up to 16 terms combined on
  // the operand load; vout (nullable, forward) receives the combined operand.
  spadj_status solve(Problem* p, int transpose, int nin, const double2* const* in, const double* a, double2* out,
                     double2* vout = nullptr) {
    if (nin < 1 || nin > 16) return p->fail(SPADJ_ERR_INVALID, "rb solve: 1..16 operand terms");
    SolveArgs S{};
    for (int t = 0; t < nin; ++t) { S.in[t] = in[t]; S.a[t] = a[t]; }
    S.vout = transpose ? nullptr : vout;
    S.nin = nin; S.out = out; S.transpose = transpose; S.phiF = ops_cur->phiT.as<double>(); S.phiA = ops_cur->phi.as<double>();
    S.Kx = Kx; S.N = N;
    const int H = 3 * N / 2;
    dim3 grid(Kx, 2, 2);
    cudaEvent_t t = p->tic();
    SPADJ_CUDA_TRY(p, launch_kernel(p->pdl, solve_kernel, grid, dim3(4 * solve_rows(H)), ssmem, p->stream, S));
    // two real H x H matvecs per pencil, each on two right-hand sides (re, im)
    p->toc(t, KC_SOLVE, 2.0 * Kx * 2.0 * H * H * 2.0);
    return check_launch(p, "rb solve");
  }

  // ---- fused column stage -------------------------------------------------------------------
  // f = Gz Y (into f), x = Phi (sum_t a_t in_t + af f) (into x), and, when expand, the six
  // grid-field columns of x into Z; one cluster of two CTAs per pencil.
  spadj_status colstep(Problem* p, double2* f, int nin, const double2* const* in, const double* a, double af,
                       double2* x, bool expand) {
    ColStepArgs S{};
    for (int q = 0; q < 3; ++q) S.yin[q] = mix(w->Y, q);
    S.gzF = gzF.as<double>();
    S.f_out = f;
    for (int t = 0; t < nin; ++t) { S.in[t] = in[t]; S.a[t] = a[t]; }
    S.nin = nin;
    S.af = af;
    S.phiF = ops_cur->phiT.as<double>();
    S.x_out = x;
    S.czE = czE.as<double>();
    S.cdzE = cdzE.as<double>();
    S.zout = expand ? w->Z.as<double2>() : nullptr;
    S.nmix = nmix;
    S.Kx = Kx; S.N = N; S.Mz = Mz;
    S.err = errbuf.as<int>();
    S.bulk = p->bulk_staging ? 1 : 0;
    const int H = 3 * N / 2;
    // algorithmic flops: fold 4 N (Mz/2) per field column, solve 2 classes x 4 H^2, expand as zflops
    const double fl = (double)Kx * (3 * 4.0 * N * (Mz / 2) + 2 * 4.0 * H * H + (expand ? 6 * 4.0 * N * (Mz / 2) : 0.0));
    cudaEvent_t t = p->tic();
    rb_colstep_kernel<<<2 * Kx, 256, csmem, p->stream>>>(S);
    p->toc(t, KC_FUSED, fl);
    return check_launch(p, "rb colstep");
  }
  // stage 1 of the step from x0: grid fields G0 of x0, f0 = F(x0), x1 = Phi(x0 + dt A10 f0) and
  // the grid fields G1 of x1
  spadj_status stage1_fused(Problem* p, const double2* x0) {
    spadj_status s = c2g_fields(p, x0, w->G0);
    if (s != SPADJ_OK) return s;
    if ((s = products_r2c(p, w->G0.as<double>())) != SPADJ_OK) return s;
    const double2* in[1] = {x0};
    double a[1] = {1.0};
    if ((s = colstep(p, st(w->f0), 1, in, a, dt * A10, st(w->x1), true)) != SPADJ_OK) return s;
    return c2r_fields(p, w->G1);
  }

  // ---- generic Runge-Kutta IMEX steps (separate kernels) ---------------------------------------
  // Stage i = 1..S of the stage equation (M + dt gam L) X_i = M X_0 + dt sum_{j<i} (A_ij F_j -
  // H_ij L X_j) in prognostic form: dt gam L X_j = S1S0 (v_j - x_j) for the solved stages (the
  // first implicit column is zero), so
  //   v_i = x_0 + sum_{j<i} dt A_ij f_j - sum_{1<=j<i} (H_ij / gam)(v_j - x_j),  x_i = Phi v_i,
  //   f_i = F(x_i) (i < S),  X_{n+1} = x_S.

  // out = sum_t a_t in_t (n >= 1); in[0] may be out itself (accumulation)
  int comb_grid() const { return (int)std::min<size_t>((ns + 255) / 256, 1024); }

  // out = sum_t a_t in_t (in[0] may be out): one launch for up to kCombMax terms
  spadj_status lincomb(Problem* p, double2* out, int n, const double2* const* in, const double* a) {
    if (n >= 1 && n <= kCombMax) {
      CombArgs A{};
      for (int t = 0; t < n; ++t) { A.in[t] = in[t]; A.a[t] = a[t]; }
      A.n = n;
      A.out = out;
      A.count = ns;
      cudaEvent_t ev = p->tic();
      SPADJ_CUDA_TRY(p, launch_kernel(p->pdl, combine_kernel, dim3(comb_grid()), dim3(256), 0, p->stream, A));
      p->toc(ev, KC_POINTWISE, 4.0 * (double)ns * (n - 1) + 2.0 * (double)ns);
      return check_launch(p, "rb combine");
    }
    int t = 0;
    bool first = true;
    while (first || t < n) {
      const double2* x0 = out;
      double a0 = 1.0;
      if (first) { x0 = in[0]; a0 = a[0]; t = 1; }
      const double2* x1 = nullptr;
      const double2* x2 = nullptr;
      double a1 = 0.0, a2 = 0.0;
      if (t < n) { x1 = in[t]; a1 = a[t]; ++t; }
      if (t < n) { x2 = in[t]; a2 = a[t]; ++t; }
      cudaEvent_t ev = p->tic();
      axpy_kernel<<<64, 256, 0, p->stream>>>(out, x0, a0, x1, a1, x2, a2, ns);
      p->toc(ev, KC_POINTWISE, 4.0 * (double)ns);
      spadj_status s = check_launch(p, "rb combine");
      if (s != SPADJ_OK) return s;
      first = false;
    }
    return SPADJ_OK;
  }

  // stage vectors of lane w: x_i (i >= 1), v_i (i >= 1), f_j (j >= 0)
  double2* gx(int i) { return st(w->rx[i - 1]); }
  double2* gv(int i) { return st(w->rv[i - 1]); }
  double2* gf(int j) { return st(w->rf[j]); }

  // terms of v_i (pointers, weights) over x_0, f_j and (v_j, x_j); the tangent's stage vectors
  // (dx_0, df_j, dv_j, dx_j) when tangent
  // out_k += c_k src for n distinct outputs (none is src), one launch
  spadj_status scatter(Problem* p, const double2* src, int n, double2* const* out, const double* c) {
    if (n == 0) return SPADJ_OK;
    ScatArgs A{};
    for (int k = 0; k < n; ++k) { A.out[k] = out[k]; A.c[k] = c[k]; }
    A.n = n;
    A.src = src;
    A.count = ns;
    cudaEvent_t ev = p->tic();
    SPADJ_CUDA_TRY(p, launch_kernel(p->pdl, scatter_kernel, dim3(comb_grid()), dim3(256), 0, p->stream, A));
    p->toc(ev, KC_POINTWISE, 4.0 * (double)ns * n);
    return check_launch(p, "rb scatter");
  }

  int stage_terms(int i, const double2* x0, const double2** in, double* a, bool tangent) {
    int n = 0;
    in[n] = x0; a[n++] = 1.0;
    for (int j = 0; j < i; ++j)
      if (tA[i][j] != 0.0) { in[n] = tangent ? st(tdf[j]) : gf(j); a[n++] = dt * tA[i][j]; }
    for (int j = 1; j < i; ++j) {
      const double h = tH[i][j] / gam;
      if (h == 0.0) continue;
      in[n] = tangent ? st(tdv[j - 1]) : gv(j); a[n++] = -h;
      in[n] = tangent ? st(tdx[j - 1]) : gx(j); a[n++] = h;
    }
    return n;
  }

  // one step x0 -> x_out (and its tangent dx0 -> dx_out when dx0 is non-null)
  spadj_status gen_step(Problem* p, const double2* x0, const double2* dx0, double2* x_out, double2* dx_out) {
    spadj_status s;
    const double one[1] = {1.0};
    if ((s = evalF(p, x0, gf(0), w->G0)) != SPADJ_OK) return s;
    if (dx0 && (s = evalJvp(p, w->G0, dx0, st(tdf[0]))) != SPADJ_OK) return s;
    for (int i = 1; i <= S; ++i) {
      const double2* in[16];
      double a[16];
      int n = stage_terms(i, x0, in, a, false);
      double2* xi = i == S ? x_out : gx(i);
      // v_i combined on the solve's operand load (and stored for the later stages and the adjoint)
      if ((s = solve(p, 0, n, in, a, xi, gv(i))) != SPADJ_OK) return s;
      if (dx0) {
        n = stage_terms(i, dx0, in, a, true);
        if ((s = lincomb(p, st(tdv[i - 1]), n, in, a)) != SPADJ_OK) return s;
        double2* dxi = i == S ? dx_out : st(tdx[i - 1]);
        const double2* v[1] = {st(tdv[i - 1])};
        if ((s = solve(p, 0, 1, v, one, dxi)) != SPADJ_OK) return s;
      }
      if (i < S) {
        if ((s = evalF(p, xi, gf(i), w->G0)) != SPADJ_OK) return s;
        if (dx0 && (s = evalJvp(p, w->G0, st(tdx[i - 1]), st(tdf[i]))) != SPADJ_OK) return s;
      }
    }
    return SPADJ_OK;
  }

  // exact reverse of gen_step: xb_in = cotangent of X_{n+1} -> xb0 = cotangent of X_n
  spadj_status gen_step_adj(Problem* p, const double2* x0, const double2* xb_in, double2* xb0) {
    spadj_status s;
    if ((s = gen_step(p, x0, nullptr, st(axs), nullptr)) != SPADJ_OK) return s;  // stage values
    const size_t sb = sizeof(double2) * ns;
    for (int i = 0; i < S; ++i) {
      SPADJ_CUDA_TRY(p, cudaMemsetAsync(afb[i].ptr, 0, sb, p->stream));  // fbar_0..fbar_{S-1}
      SPADJ_CUDA_TRY(p, cudaMemsetAsync(axb[i].ptr, 0, sb, p->stream));  // xbar_1..xbar_{S-1}
      SPADJ_CUDA_TRY(p, cudaMemsetAsync(avb[i].ptr, 0, sb, p->stream));  // vbar_1..vbar_S
    }
    SPADJ_CUDA_TRY(p, cudaMemsetAsync(aacc.ptr, 0, sb, p->stream));
    const double one[1] = {1.0};
    for (int i = S; i >= 1; --i) {
      double2* xbi = i == S ? const_cast<double2*>(xb_in) : st(axb[i - 1]);
      if (i < S && nonlinear) {  // xbar_i += (dF/dx)(x_i)^H fbar_i
        if ((s = c2g_fields(p, gx(i), w->G0)) != SPADJ_OK) return s;
        const double2* fb[1] = {st(afb[i])};
        const double2* ad[1] = {xbi};
        if ((s = evalVjp(p, w->G0, 1, fb, one, 1, ad, one, xbi)) != SPADJ_OK) return s;
      }
      double2* vbi = st(avb[i - 1]);
      { const double2* v[1] = {xbi};  // vbar_i += Phi^H xbar_i
        if ((s = solve(p, 1, 1, v, one, st(atmp))) != SPADJ_OK) return s; }
      { const double2* in[2] = {vbi, st(atmp)}; const double a[2] = {1.0, 1.0};
        if ((s = lincomb(p, vbi, 2, in, a)) != SPADJ_OK) return s; }
      // v_i = x_0 + sum_j dt A_ij f_j - sum_j h_ij (v_j - x_j): distribute vbar_i, every cotangent
      // it reaches in one launch
      {
        double2* outs[kCombMax];
        double cs[kCombMax];
        int no = 0;
        outs[no] = st(aacc); cs[no++] = 1.0;
        for (int j = 0; j < i; ++j)
          if (tA[i][j] != 0.0) { outs[no] = st(afb[j]); cs[no++] = dt * tA[i][j]; }
        for (int j = 1; j < i; ++j) {
          const double h = tH[i][j] / gam;
          if (h == 0.0) continue;
          outs[no] = st(avb[j - 1]); cs[no++] = -h;
          outs[no] = st(axb[j - 1]); cs[no++] = h;
        }
        if ((s = scatter(p, vbi, no, outs, cs)) != SPADJ_OK) return s;
      }
    }
    // xbar_0 = acc + (dF/dx)(x_0)^H fbar_0
    if (nonlinear && (s = c2g_fields(p, x0, w->G0)) != SPADJ_OK) return s;
    const double2* fb[1] = {st(afb[0])};
    const double2* ad[1] = {st(aacc)};
    return evalVjp(p, w->G0, 1, fb, one, 1, ad, one, xb0);
  }

  // ---- RK222 steps ---------------------------------------------------------------------------
  bool use_fused(Problem* p) const { return fused && p->fuse_columns; }

  spadj_status step_fwd(Problem* p, const double2* x0, double2* x2) {
    if (generic) return gen_step(p, x0, nullptr, x2, nullptr);
    if (use_fused(p)) {
      spadj_status s = stage1_fused(p, x0);
      if (s != SPADJ_OK) return s;
      if ((s = products_r2c(p, w->G1.as<double>())) != SPADJ_OK) return s;
      const double2* in[3] = {x0, st(w->f0), st(w->x1)};
      double a[3] = {1.0 - cc, dt * (A20 - cc * A10), cc};
      return colstep(p, st(w->f1), 3, in, a, dt * A21, x2, false);
    }
    spadj_status s;
    if ((s = evalF(p, x0, st(w->f0), w->G0)) != SPADJ_OK) return s;
    { const double2* in[2] = {x0, st(w->f0)}; double a[2] = {1.0, dt * A10};
      if ((s = solve(p, 0, 2, in, a, st(w->x1))) != SPADJ_OK) return s; }
    if ((s = evalF(p, st(w->x1), st(w->f1), w->G1)) != SPADJ_OK) return s;
    const double2* in[4] = {x0, st(w->f0), st(w->f1), st(w->x1)};
    double a[4] = {1.0 - cc, dt * (A20 - cc * A10), dt * A21, cc};
    return solve(p, 0, 4, in, a, x2);
  }

  spadj_status step_tan(Problem* p, const double2* x0, const double2* dx0, double2* x2, double2* dx2) {
    if (generic) return gen_step(p, x0, dx0, x2, dx2);
    spadj_status s;
    if ((s = evalF(p, x0, st(w->f0), w->G0)) != SPADJ_OK) return s;
    if ((s = evalJvp(p, w->G0, dx0, st(df0))) != SPADJ_OK) return s;
    { const double2* in[2] = {x0, st(w->f0)}; double a[2] = {1.0, dt * A10};
      if ((s = solve(p, 0, 2, in, a, st(w->x1))) != SPADJ_OK) return s; }
    { const double2* in[2] = {dx0, st(df0)}; double a[2] = {1.0, dt * A10};
      if ((s = solve(p, 0, 2, in, a, st(dx1))) != SPADJ_OK) return s; }
    if ((s = evalF(p, st(w->x1), st(w->f1), w->G1)) != SPADJ_OK) return s;
    if ((s = evalJvp(p, w->G1, st(dx1), st(df1))) != SPADJ_OK) return s;
    double a[4] = {1.0 - cc, dt * (A20 - cc * A10), dt * A21, cc};
    { const double2* in[4] = {x0, st(w->f0), st(w->f1), st(w->x1)};
      if ((s = solve(p, 0, 4, in, a, x2)) != SPADJ_OK) return s; }
    const double2* in[4] = {dx0, st(df0), st(df1), st(dx1)};
    return solve(p, 0, 4, in, a, dx2);
  }

  // xb0 = cotangent of X_n from xb2 = cotangent of X_{n+1}, primal x0 = X_n.
  spadj_status step_adj(Problem* p, const double2* x0, const double2* xb2, double2* xb0) {
    if (generic) return gen_step_adj(p, x0, xb2, xb0);
    spadj_status s;
    // the transposed stage-2 solve does not depend on the stage recomputation: it runs on the
    // second internal stream and overlaps it
    SPADJ_CUDA_TRY(p, cudaEventRecord(evFork, p->stream));
    SPADJ_CUDA_TRY(p, cudaStreamWaitEvent(gs2, evFork, 0));
    {
      cudaStream_t main = p->stream;
      p->stream = gs2;
      const double2* in[1] = {xb2};
      double a[1] = {1.0};
      s = solve(p, 1, 1, in, a, st(vb2));
      p->stream = main;
      if (s != SPADJ_OK) return s;
    }
    SPADJ_CUDA_TRY(p, cudaEventRecord(evJoin, gs2));
    if (use_fused(p)) {
      if ((s = stage1_fused(p, x0)) != SPADJ_OK) return s;
    } else {
      if ((s = evalF(p, x0, st(w->f0), w->G0)) != SPADJ_OK) return s;
      { const double2* in[2] = {x0, st(w->f0)}; double a[2] = {1.0, dt * A10};
        if ((s = solve(p, 0, 2, in, a, st(w->x1))) != SPADJ_OK) return s; }
      if (nonlinear && (s = c2g_fields(p, st(w->x1), w->G1)) != SPADJ_OK) return s;
    }
    SPADJ_CUDA_TRY(p, cudaStreamWaitEvent(p->stream, evJoin, 0));
    if (use_fused(p)) {
      // xb1 = c vb2 + (dF/dx1)^dagger (dt A21 vb2); vb1 = Phi^H xb1; then the first transform
      // of the second product, Gz^T (dt(A20 - c A10) vb2 + dt A10 vb1), in the same cluster kernel
      { const double2* fb[1] = {st(vb2)}; double al[1] = {dt * A21};
        if ((s = vjp_expand(p, 1, fb, al)) != SPADJ_OK) return s; }
      if ((s = vjp_middle(p, w->G1)) != SPADJ_OK) return s;
      { const double2* ad[1] = {st(vb2)}; double be[1] = {cc};
        if ((s = colstepT(p, 1, ad, be, st(vb1), st(vb2), dt * (A20 - cc * A10), dt * A10)) != SPADJ_OK) return s; }
      if ((s = vjp_middle(p, w->G0)) != SPADJ_OK) return s;
      const double2* ad[2] = {st(vb2), st(vb1)};
      double be[2] = {1.0 - cc, 1.0};
      return vjp_fold(p, 2, ad, be, xb0);
    }
    // xb1 = c vb2 + (dF/dx1)^dagger (dt A21 vb2)
    { const double2* fb[1] = {st(vb2)}; double al[1] = {dt * A21};
      const double2* ad[1] = {st(vb2)}; double be[1] = {cc};
      if ((s = evalVjp(p, w->G1, 1, fb, al, 1, ad, be, st(xb1))) != SPADJ_OK) return s; }
    { const double2* in[1] = {st(xb1)}; double a[1] = {1.0};
      if ((s = solve(p, 1, 1, in, a, st(vb1))) != SPADJ_OK) return s; }
    // xb0 = (1-c) vb2 + vb1 + (dF/dx0)^dagger (dt(A20 - c A10) vb2 + dt A10 vb1)
    const double2* fb[2] = {st(vb2), st(vb1)};
    double al[2] = {dt * (A20 - cc * A10), dt * A10};
    const double2* ad[2] = {st(vb2), st(vb1)};
    double be[2] = {1.0 - cc, 1.0};
    return evalVjp(p, w->G0, 2, fb, al, 2, ad, be, xb0);
  }

  // The fused adjoint step with its stage-1 grid fields (G0 of X_n, G1 of the stage value x1)
  // already computed into sg by stage1_fused on another lane: the same kernels on the same data as
  // step_adj, without the recomputation on the critical path.
  spadj_status step_adj_staged(Problem* p, WS& sg, const double2* xb2, double2* xb0) {
    spadj_status s;
    { const double2* in[1] = {xb2}; double a[1] = {1.0};
      if ((s = solve(p, 1, 1, in, a, st(vb2))) != SPADJ_OK) return s; }
    { const double2* fb[1] = {st(vb2)}; double al[1] = {dt * A21};
      if ((s = vjp_expand(p, 1, fb, al)) != SPADJ_OK) return s; }
    if ((s = vjp_middle(p, sg.G1)) != SPADJ_OK) return s;
    { const double2* ad[1] = {st(vb2)}; double be[1] = {cc};
      if ((s = colstepT(p, 1, ad, be, st(vb1), st(vb2), dt * (A20 - cc * A10), dt * A10)) != SPADJ_OK) return s; }
    if ((s = vjp_middle(p, sg.G0)) != SPADJ_OK) return s;
    const double2* ad[2] = {st(vb2), st(vb1)};
    double be[2] = {1.0 - cc, 1.0};
    return vjp_fold(p, 2, ad, be, xb0);
  }

  // ---- C-ABI operations ----------------------------------------------------------------------
  spadj_status transform(Problem* p, int kind, const double* in, double* out) override {
    // one scalar field: coefficients [Kx][N] <-> grid [Mz][Mx]
    const double2* ci = reinterpret_cast<const double2*>(in);
    double2* co = reinterpret_cast<double2*>(out);
    spadj_status s;
    if (kind == 0 || kind == 3) {
      ZJobs zj{};
      zj.expand = 1;
      zj.j[0] = zexpand(ci, kind == 0 ? czE.as<double>() : gzTE.as<double>(), 0, mix(w->Z, 0));
      zj.n = 1;
      if ((s = launch_z(p, zj)) != SPADJ_OK) return s;
      XJobs xj{};
      xj.j[0] = kind == 0 ? xc2r(mix(w->Z, 0), 0, 1.0, 1.0, out) : xc2r(mix(w->Z, 0), 0, 1.0 / Mx, 0.5 / Mx, out);
      xj.n = 1;
      return launch_x(p, xj);
    }
    if (kind == 1 || kind == 2) {
      XJobs xj{};
      xj.j[0] = kind == 1 ? xr2c(in, 0, nullptr, 0, 1.0 / Mx, 1.0 / Mx, mix(w->Y, 0))
                          : xr2c(in, 0, nullptr, 0, 1.0, 2.0, mix(w->Y, 0));
      xj.n = 1;
      if ((s = launch_x(p, xj)) != SPADJ_OK) return s;
      ZJobs zj{};
      zj.expand = 0;
      zj.j[0] = zfold(mix(w->Y, 0), kind == 1 ? gzF.as<double>() : czTF.as<double>(), 0, co);
      zj.n = 1;
      return launch_z(p, zj);
    }
    return p->fail(SPADJ_ERR_INVALID, "transform: kind must be 0..3");
  }

  // Same transform as transform() above, with the intermediate mixed array supplied by the
  // caller (the no-allocation entry point passes its static device scratch here).
  spadj_status transform_into(Problem* p, int kind, const double* in, double* out, double2* scratch) {
    const double2* ci = reinterpret_cast<const double2*>(in);
    double2* co = reinterpret_cast<double2*>(out);
    spadj_status s;
    if (kind == 0 || kind == 3) {
      ZJobs zj{};
      zj.expand = 1;
      zj.j[0] = zexpand(ci, kind == 0 ? czE.as<double>() : gzTE.as<double>(), 0, scratch);
      zj.n = 1;
      if ((s = launch_z(p, zj)) != SPADJ_OK) return s;
      XJobs xj{};
      xj.j[0] = kind == 0 ? xc2r(scratch, 0, 1.0, 1.0, out) : xc2r(scratch, 0, 1.0 / Mx, 0.5 / Mx, out);
      xj.n = 1;
      return launch_x(p, xj);
    }
    if (kind == 1 || kind == 2) {
      XJobs xj{};
      xj.j[0] = kind == 1 ? xr2c(in, 0, nullptr, 0, 1.0 / Mx, 1.0 / Mx, scratch)
                          : xr2c(in, 0, nullptr, 0, 1.0, 2.0, scratch);
      xj.n = 1;
      if ((s = launch_x(p, xj)) != SPADJ_OK) return s;
      ZJobs zj{};
      zj.expand = 0;
      zj.j[0] = zfold(scratch, kind == 1 ? gzF.as<double>() : czTF.as<double>(), 0, co);
      zj.n = 1;
      return launch_z(p, zj);
    }
    return p->fail(SPADJ_ERR_INVALID, "transform_noalloc: kind must be 0..3");
  }

  spadj_status eval_F(Problem* p, int mode, const double* x, const double* dx, double* out) override {
    const double2* xc = reinterpret_cast<const double2*>(x);
    const double2* dc = reinterpret_cast<const double2*>(dx);
    double2* oc = reinterpret_cast<double2*>(out);
    spadj_status s;
    if (mode == 0) return evalF(p, xc, oc, w->G0);
    if ((s = c2g_fields(p, xc, w->G0)) != SPADJ_OK) return s;
    if (mode == 1) return evalJvp(p, w->G0, dc, oc);
    const double2* fb[1] = {dc};
    double al[1] = {1.0};
    return evalVjp(p, w->G0, 1, fb, al, 0, nullptr, nullptr, oc);
  }

  spadj_status pencil_solve(Problem* p, int transpose, const double* v, double* x) {
    select_base();  // the stage operator of the descriptor's dt
    const double2* in[1] = {reinterpret_cast<const double2*>(v)};
    double a[1] = {1.0};
    return solve(p, transpose, 1, in, a, reinterpret_cast<double2*>(x));
  }

  // Run the library's work on its internal stream, ordered after the caller's stream on
  // entry and before it on exit.
  struct StreamScope {
    RB* r;
    Problem* p;
    cudaStream_t us;
    StreamScope(RB* r_, Problem* p_) : r(r_), p(p_), us(p_->stream) {
      cudaEventRecord(r->evIn, us);
      cudaStreamWaitEvent(r->gs, r->evIn, 0);
      p->stream = r->gs;
    }
    ~StreamScope() {
      cudaEventRecord(r->evOut, r->gs);
      cudaStreamWaitEvent(us, r->evOut, 0);
      p->stream = us;
    }
  };

  bool use_graphs(Problem* p) const { return !p->timing.enabled; }

  spadj_status capture(Problem* p, cudaGraphExec_t* exec, const std::function<spadj_status()>& body) {
    SPADJ_CUDA_TRY(p, cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    spadj_status s = body();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->stream, &g);
    if (s != SPADJ_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return p->fail(SPADJ_ERR_CUDA, std::string("rb: graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return p->fail(SPADJ_ERR_CUDA, std::string("rb: graph instantiate: ") + cudaGetErrorString(e));
    return SPADJ_OK;
  }

  // one forward step Sb[ci] -> Sb[1-ci] (captured graph when timing is off)
  spadj_status run_fwd(Problem* p, int ci) {
    double2* x0 = Sb[ci];
    double2* x2 = Sb[1 - ci];
    if (!use_graphs(p)) return step_fwd(p, x0, x2);
    if (!ops_cur->gFwd[ci]) {
      spadj_status s = capture(p, &ops_cur->gFwd[ci], [&] { return step_fwd(p, x0, x2); });
      if (s != SPADJ_OK) return s;
    }
    SPADJ_CUDA_TRY(p, cudaGraphLaunch(ops_cur->gFwd[ci], p->stream));
    return SPADJ_OK;
  }

  // one forward step of lane 1 (stream gsB, workspace ws[1]): SbB[ci] -> SbB[1-ci]
  spadj_status run_fwd_lane1(Problem* p, int ci) {
    cudaStream_t main = p->stream;
    p->stream = gsB;
    w = &ws[1];
    double2* x0 = SbB[ci];
    double2* x2 = SbB[1 - ci];
    spadj_status s = SPADJ_OK;
    if (!use_graphs(p)) {
      s = step_fwd(p, x0, x2);
    } else {
      if (!ops_cur->gFwdB[ci]) s = capture(p, &ops_cur->gFwdB[ci], [&] { return step_fwd(p, x0, x2); });
      if (s == SPADJ_OK) {
        cudaError_t e = cudaGraphLaunch(ops_cur->gFwdB[ci], p->stream);
        if (e != cudaSuccess) s = p->fail(SPADJ_ERR_CUDA, std::string("rb: graph launch: ") + cudaGetErrorString(e));
      }
    }
    w = &ws[0];
    p->stream = main;
    return s;
  }

  // one adjoint step at state Sb[ci]: Yb[yi] (cotangent of X_{n+1}) -> Yb[1-yi] (of X_n)
  spadj_status run_adj(Problem* p, int ci, int yi) {
    const double2* x0 = Sb[ci];
    const double2* xb2 = Yb[yi];
    double2* xb0 = Yb[1 - yi];
    if (!use_graphs(p)) return step_adj(p, x0, xb2, xb0);
    if (!ops_cur->gAdj[ci][yi]) {
      spadj_status s = capture(p, &ops_cur->gAdj[ci][yi], [&] { return step_adj(p, x0, xb2, xb0); });
      if (s != SPADJ_OK) return s;
    }
    SPADJ_CUDA_TRY(p, cudaGraphLaunch(ops_cur->gAdj[ci][yi], p->stream));
    return SPADJ_OK;
  }

  // lane 2 (stream gsC, workspace ws[2 + c]): stage 1 of the step from Sb[c] (grid fields for the
  // staged adjoint step)
  spadj_status run_stage_lane2(Problem* p, int c) {
    cudaStream_t main = p->stream;
    p->stream = gsC;
    w = &ws[2 + c];
    spadj_status s = SPADJ_OK;
    const double2* x0 = Sb[c];
    if (!use_graphs(p)) {
      s = stage1_fused(p, x0);
    } else {
      if (!ops_cur->gStage[c]) s = capture(p, &ops_cur->gStage[c], [&] { return stage1_fused(p, x0); });
      if (s == SPADJ_OK) {
        cudaError_t e = cudaGraphLaunch(ops_cur->gStage[c], p->stream);
        if (e != cudaSuccess) s = p->fail(SPADJ_ERR_CUDA, std::string("rb: graph launch: ") + cudaGetErrorString(e));
      }
    }
    w = &ws[0];
    p->stream = main;
    return s;
  }

  // lane 0: staged adjoint step with the grid fields of ws[2 + c]: Yb[yi] -> Yb[1 - yi]
  spadj_status run_adj_staged(Problem* p, int c, int yi) {
    WS& sg = ws[2 + c];
    const double2* xb2 = Yb[yi];
    double2* xb0 = Yb[1 - yi];
    if (!use_graphs(p)) return step_adj_staged(p, sg, xb2, xb0);
    if (!ops_cur->gAdjS[c][yi]) {
      spadj_status s = capture(p, &ops_cur->gAdjS[c][yi], [&] { return step_adj_staged(p, sg, xb2, xb0); });
      if (s != SPADJ_OK) return s;
    }
    SPADJ_CUDA_TRY(p, cudaGraphLaunch(ops_cur->gAdjS[c][yi], p->stream));
    return SPADJ_OK;
  }

  spadj_status forward(Problem* p, int n_steps, const double* x0, double* x_out, double* traj) override {
    if (n_steps < 0) return p->fail(SPADJ_ERR_INVALID, "forward: n_steps < 0");
    spadj_status ps = prepare_steps(p, n_steps);
    if (ps != SPADJ_OK) return ps;
    const size_t sb = sizeof(double2) * ns;
    StreamScope scope(this, p);
    int ci = 0;
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(Sb[ci], x0, sb, cudaMemcpyDeviceToDevice, p->stream));
    if (traj) SPADJ_CUDA_TRY(p, cudaMemcpyAsync(traj, x0, sb, cudaMemcpyDeviceToDevice, p->stream));
    for (int n = 0; n < n_steps; ++n) {
      spadj_status s = select_step(p, n);
      if (s == SPADJ_OK) s = run_fwd(p, ci);
      select_base();
      if (s != SPADJ_OK) return s;
      ci = 1 - ci;
      if (traj)
        SPADJ_CUDA_TRY(p, cudaMemcpyAsync(traj + (size_t)(n + 1) * 2 * ns, Sb[ci], sb, cudaMemcpyDeviceToDevice, p->stream));
    }
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(x_out, Sb[ci], sb, cudaMemcpyDeviceToDevice, p->stream));
    return SPADJ_OK;
  }

  spadj_status tangent(Problem* p, int n_steps, const double* x0, const double* dx0, double* dx_out) override {
    if (n_steps < 0) return p->fail(SPADJ_ERR_INVALID, "tangent: n_steps < 0");
    spadj_status ps = prepare_steps(p, n_steps);
    if (ps != SPADJ_OK) return ps;
    const size_t sb = sizeof(double2) * ns;
    StreamScope scope(this, p);
    double2* T[2] = {tmpx.as<double2>(), tmpy.as<double2>()};
    int ci = 0;
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(Sb[ci], x0, sb, cudaMemcpyDeviceToDevice, p->stream));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(T[ci], dx0, sb, cudaMemcpyDeviceToDevice, p->stream));
    for (int n = 0; n < n_steps; ++n) {
      spadj_status s = select_step(p, n);
      if (s == SPADJ_OK) s = step_tan(p, Sb[ci], T[ci], Sb[1 - ci], T[1 - ci]);
      select_base();
      if (s != SPADJ_OK) return s;
      ci = 1 - ci;
    }
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(dx_out, T[ci], sb, cudaMemcpyDeviceToDevice, p->stream));
    return SPADJ_OK;
  }

  spadj_status adjoint(Problem* p, int n_steps, const double* traj, const double* y_final, double* grad,
                       double* grad_p) override {
    if (n_steps < 1) return p->fail(SPADJ_ERR_INVALID, "adjoint: n_steps < 1");
    if (grad_p) return p->fail(SPADJ_ERR_INVALID, "rb: the problem has no parameters (grad_p must be NULL)");
    spadj_status ps = prepare_steps(p, n_steps);
    if (ps != SPADJ_OK) return ps;
    const size_t sb = sizeof(double2) * ns;
    StreamScope scope(this, p);
    int yi = 0;
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(Yb[yi], y_final, sb, cudaMemcpyDeviceToDevice, p->stream));
    for (int n = n_steps - 1; n >= 0; --n) {
      const double2* xn = reinterpret_cast<const double2*>(traj) + (size_t)n * ns;
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(Sb[0], xn, sb, cudaMemcpyDeviceToDevice, p->stream));
      spadj_status s = select_step(p, n);
      if (s == SPADJ_OK) s = run_adj(p, 0, yi);
      select_base();
      if (s != SPADJ_OK) return s;
      yi = 1 - yi;
    }
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(grad, Yb[yi], sb, cudaMemcpyDeviceToDevice, p->stream));
    return SPADJ_OK;
  }

  // ---- one step at a time (the same step graphs as the sweeps) -------------------------------
  // Runge-Kutta schemes restart from X_n alone, and the adjoint state is the cotangent of X_n.
  int step_blocks(int which) const override { (void)which; return 1; }

  // operators of step n's size (built on first use)
  spadj_status prepare_step(Problem* p, int n) {
    if (n < 0) return p->fail(SPADJ_ERR_INVALID, "step: n < 0");
    if (sched.empty()) return SPADJ_OK;
    if (n >= (int)sched.size()) return p->fail(SPADJ_ERR_INVALID, "rb: step index beyond the step-size schedule");
    OpSet* os = nullptr;
    return opset_for(p, sched[n], &os);
  }

  spadj_status step_forward(Problem* p, int n, const double* s_n, double* s_np1) override {
    spadj_status s = prepare_step(p, n);
    if (s != SPADJ_OK) return s;
    const size_t sb = sizeof(double2) * ns;
    StreamScope scope(this, p);
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(Sb[0], s_n, sb, cudaMemcpyDeviceToDevice, p->stream));
    s = select_step(p, n);
    if (s == SPADJ_OK) s = run_fwd(p, 0);
    select_base();
    if (s != SPADJ_OK) return s;
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(s_np1, Sb[1], sb, cudaMemcpyDeviceToDevice, p->stream));
    return SPADJ_OK;
  }

  spadj_status step_tangent(Problem* p, int n, const double* s_n, const double* ds_n, double* ds_np1) override {
    spadj_status s = prepare_step(p, n);
    if (s != SPADJ_OK) return s;
    const size_t sb = sizeof(double2) * ns;
    StreamScope scope(this, p);
    double2* T[2] = {tmpx.as<double2>(), tmpy.as<double2>()};
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(Sb[0], s_n, sb, cudaMemcpyDeviceToDevice, p->stream));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(T[0], ds_n, sb, cudaMemcpyDeviceToDevice, p->stream));
    s = select_step(p, n);
    if (s == SPADJ_OK) s = step_tan(p, Sb[0], T[0], Sb[1], T[1]);
    select_base();
    if (s != SPADJ_OK) return s;
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(ds_np1, T[1], sb, cudaMemcpyDeviceToDevice, p->stream));
    return SPADJ_OK;
  }

  // y_n = (dX_{n+1}/dX_n)^dagger y_{n+1} + src; y_{n+1} = NULL stands for a zero cotangent (then
  // y_n = src, the seed of a reverse sweep at the final state).
  spadj_status step_adjoint(Problem* p, int n, const double* x_n, const double* y_np1, const double* src, double* y_n,
                            double* gp_accum) override {
    if (gp_accum) return p->fail(SPADJ_ERR_INVALID, "rb: the problem has no parameters (gp_accum must be NULL)");
    const size_t sb = sizeof(double2) * ns;
    if (!y_np1) {
      if (src) SPADJ_CUDA_TRY(p, cudaMemcpyAsync(y_n, src, sb, cudaMemcpyDeviceToDevice, p->stream));
      else SPADJ_CUDA_TRY(p, cudaMemsetAsync(y_n, 0, sb, p->stream));
      return SPADJ_OK;
    }
    spadj_status s = prepare_step(p, n);
    if (s != SPADJ_OK) return s;
    StreamScope scope(this, p);
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(Sb[0], x_n, sb, cudaMemcpyDeviceToDevice, p->stream));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(Yb[0], y_np1, sb, cudaMemcpyDeviceToDevice, p->stream));
    s = select_step(p, n);
    if (s == SPADJ_OK) s = run_adj(p, 0, 0);
    select_base();
    if (s != SPADJ_OK) return s;
    if (src) {  // the injection of the checkpointed sweep
      axpy_kernel<<<64, 256, 0, p->stream>>>(Yb[1], Yb[1], 1.0, reinterpret_cast<const double2*>(src), 1.0, nullptr,
                                             0.0, ns);
      if ((s = check_launch(p, "rb step src")) != SPADJ_OK) return s;
    }
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(y_n, Yb[1], sb, cudaMemcpyDeviceToDevice, p->stream));
    return SPADJ_OK;
  }

  spadj_status objective(Problem* p, int objective, const double* obj_data, const double* x, double* J_dev,
                         double* sd) override {
    (void)obj_data;
    if (objective != SPADJ_OBJ_ENERGY) return p->fail(SPADJ_ERR_UNSUPPORTED, "rb: objective must be ENERGY");
    cudaEvent_t t = p->tic();
    energy_kernel<<<Kx, 128, 0, p->stream>>>(reinterpret_cast<const double2*>(x), gmat.as<double>(), Lx, Kx, N,
                                             partial.as<double>(), reinterpret_cast<double2*>(sd));
    p->toc(t, KC_OBJECTIVE, 8.0 * Kx * 2 * N * N);
    spadj_status s = check_launch(p, "rb energy");
    if (s != SPADJ_OK) return s;
    sum_kernel<<<1, 128, 0, p->stream>>>(partial.as<double>(), Kx, J_dev);
    return check_launch(p, "rb sum");
  }

  int last_recompute = 0;

  // Checkpointed reverse sweep.  objective_kind >= 0: seed dJ/dX_N from the objective kernel
  // (J to J_host).  objective_kind < 0: seeds supplied by the caller, seed_at[n] = index into
  // `seeds` ([n_seeds][state], device) of the cotangent injected at X_n, or -1.
  //
  // Lanes run the binomial schedule concurrently: lane 1 (stream gsB, workspace ws[1]) executes
  // the forward sweep, every recomputation and the checkpoint copies; lane 0 (the problem's
  // internal stream) the objective and the adjoint steps.  The state X_k for the adjoint step k
  // moves from lane 1 into the staging buffer Sb[k % 2], so lane 1 recomputes the states of the
  // next adjoint step while lane 0 is still reversing step k.  With the fused scheme a third lane
  // (stream gsC) takes X_k from Sb[k % 2] and recomputes the stage-1 grid fields of step k into
  // ws[2 + k % 2], and lane 0 runs only the rest of the adjoint step (step_adj_staged): the
  // recomputation leaves the critical path.  Events: evCopied[c] (X_k in Sb[c]), evStaged[c]
  // (grid fields in ws[2 + c], Sb[c] free), evAdj[c] (the adjoint step that read ws[2 + c] or
  // Sb[c] is done).
  spadj_status reverse(Problem* p, const double* x0, int n_steps, int ckpt_slots, int objective_kind,
                       const double* obj_data, const std::vector<int>& seed_at, const double* seeds, double* J_host,
                       double* grad) {
    if (n_steps < 1) return p->fail(SPADJ_ERR_INVALID, "gradient: n_steps < 1");
    if (objective_kind >= 0 && objective_kind != SPADJ_OBJ_ENERGY)
      return p->fail(SPADJ_ERR_UNSUPPORTED, "rb: objective must be ENERGY");
    {
      spadj_status ps = prepare_steps(p, n_steps);
      if (ps != SPADJ_OK) return ps;
    }
    int S = (ckpt_slots <= 0 || ckpt_slots > n_steps + 1) ? n_steps + 1 : ckpt_slots;
    const size_t sb = sizeof(double2) * ns;
    SPADJ_CUDA_TRY(p, slots.ensure(sb * (size_t)S));
    CkptPlanner planner;
    const int H = std::min(p->host_slots, n_steps);
    std::vector<CkptOp> ops = H > 0 ? planner.plan2(n_steps, S, H) : planner.plan(n_steps, S);
    if (H > 0) SPADJ_CUDA_TRY(p, hslots.ensure(sb * (size_t)H));
    StreamScope scope(this, p);
    const bool staged = use_fused(p);
    SPADJ_CUDA_TRY(p, cudaEventRecord(evFree, p->stream));
    SPADJ_CUDA_TRY(p, cudaStreamWaitEvent(gsB, evFree, 0));
    SPADJ_CUDA_TRY(p, cudaStreamWaitEvent(gsC, evFree, 0));
    int ciB = 0, yi = 0;
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(SbB[ciB], x0, sb, cudaMemcpyDeviceToDevice, gsB));
    int cur_step = 0;
    int recompute = 0;
    bool have_seed = false;
    // device slots 0..S-1, host slots S..S+H-1
    auto slot_ptr = [&](int sl) {
      return sl < S ? slots.as<char>() + (size_t)sl * sb : hslots.as<char>() + (size_t)(sl - S) * sb;
    };
    auto seed_ptr = [&](int n) -> const double2* {
      if (objective_kind >= 0 || n < 0 || n >= (int)seed_at.size() || seed_at[n] < 0) return nullptr;
      return reinterpret_cast<const double2*>(seeds) + (size_t)seed_at[n] * ns;
    };
    // X_k (current state of lane 1) -> Sb[k % 2] for lane 0 (main_reads) or lane 2
    auto handoff = [&](int k, bool main_reads) -> spadj_status {
      const int c = k & 1;
      SPADJ_CUDA_TRY(p, cudaStreamWaitEvent(gsB, evAdj[c], 0));  // the step that last read Sb[c] is done
      if (staged) SPADJ_CUDA_TRY(p, cudaStreamWaitEvent(gsB, evStaged[c], 0));  // lane 2 has read Sb[c]
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(Sb[c], SbB[ciB], sb, cudaMemcpyDeviceToDevice, gsB));
      SPADJ_CUDA_TRY(p, cudaEventRecord(evCopied[c], gsB));
      if (main_reads) SPADJ_CUDA_TRY(p, cudaStreamWaitEvent(p->stream, evCopied[c], 0));
      return SPADJ_OK;
    };
    for (const CkptOp& op : ops) {
      spadj_status s = SPADJ_OK;
      switch (op.type) {
        case CK_STORE:
          SPADJ_CUDA_TRY(p, cudaMemcpyAsync(slot_ptr(op.slot), SbB[ciB], sb,
                                            op.slot < S ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, gsB));
          break;
        case CK_RESTORE:
          if (cur_step != op.a) {
            SPADJ_CUDA_TRY(p, cudaMemcpyAsync(SbB[ciB], slot_ptr(op.slot), sb,
                                              op.slot < S ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, gsB));
            cur_step = op.a;
          }
          break;
        case CK_ADVANCE:
          for (int k = op.a; k < op.b; ++k) {
            s = select_step(p, k);
            if (s == SPADJ_OK) s = run_fwd_lane1(p, ciB);
            select_base();
            if (s != SPADJ_OK) return s;
            ciB = 1 - ciB;
            ++recompute;
          }
          cur_step = op.b;
          break;
        case CK_OBJECTIVE:
          if ((s = handoff(n_steps, true)) != SPADJ_OK) return s;
          if (objective_kind >= 0) {
            if ((s = objective(p, objective_kind, obj_data, reinterpret_cast<const double*>(Sb[n_steps & 1]),
                               Jdev.as<double>(), reinterpret_cast<double*>(Yb[yi]))) != SPADJ_OK)
              return s;
          } else if (const double2* sp = seed_ptr(n_steps)) {
            SPADJ_CUDA_TRY(p, cudaMemcpyAsync(Yb[yi], sp, sb, cudaMemcpyDeviceToDevice, p->stream));
          } else {
            SPADJ_CUDA_TRY(p, cudaMemsetAsync(Yb[yi], 0, sb, p->stream));
          }
          SPADJ_CUDA_TRY(p, cudaEventRecord(evAdj[n_steps & 1], p->stream));
          have_seed = true;
          break;
        case CK_ADJOINT: {
          if (!have_seed) return p->fail(SPADJ_ERR_INVALID, "gradient: schedule reached an adjoint step before the objective");
          const int c = op.a & 1;
          if ((s = handoff(op.a, !staged)) != SPADJ_OK) return s;
          s = select_step(p, op.a);
          if (s == SPADJ_OK && staged) {
            // lane 2: stage 1 of step a from Sb[c] into ws[2 + c], once lane 0 has finished the
            // adjoint step that last read ws[2 + c]
            cudaError_t e = cudaStreamWaitEvent(gsC, evCopied[c], 0);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(gsC, evAdj[c], 0);
            if (e != cudaSuccess) s = p->fail(SPADJ_ERR_CUDA, std::string("rb: lane 2 wait: ") + cudaGetErrorString(e));
            if (s == SPADJ_OK) s = run_stage_lane2(p, c);
            if (s == SPADJ_OK) {
              e = cudaEventRecord(evStaged[c], gsC);
              if (e == cudaSuccess) e = cudaStreamWaitEvent(p->stream, evStaged[c], 0);
              if (e != cudaSuccess) s = p->fail(SPADJ_ERR_CUDA, std::string("rb: lane 2 event: ") + cudaGetErrorString(e));
            }
            if (s == SPADJ_OK) s = run_adj_staged(p, c, yi);
          } else if (s == SPADJ_OK) {
            s = run_adj(p, c, yi);
          }
          select_base();
          if (s != SPADJ_OK) return s;
          SPADJ_CUDA_TRY(p, cudaEventRecord(evAdj[c], p->stream));
          yi = 1 - yi;
          if (const double2* sp = seed_ptr(op.a)) {  // cotangent injected at X_a
            axpy_kernel<<<64, 256, 0, p->stream>>>(Yb[yi], Yb[yi], 1.0, sp, 1.0, nullptr, 0.0, ns);
            if ((s = check_launch(p, "rb seed")) != SPADJ_OK) return s;
          }
          break;
        }
        default:
          break;
      }
    }
    last_recompute = recompute;
    SPADJ_CUDA_TRY(p, cudaEventRecord(evBdone, gsB));
    SPADJ_CUDA_TRY(p, cudaStreamWaitEvent(p->stream, evBdone, 0));
    SPADJ_CUDA_TRY(p, cudaEventRecord(evCdone, gsC));
    SPADJ_CUDA_TRY(p, cudaStreamWaitEvent(p->stream, evCdone, 0));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(grad, Yb[yi], sb, cudaMemcpyDeviceToDevice, p->stream));
    if (J_host && objective_kind >= 0) {
      int err = 0;
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(J_host, Jdev.ptr, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(&err, errbuf.ptr, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
      SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
      if (err) {
        SPADJ_CUDA_TRY(p, cudaMemsetAsync(errbuf.ptr, 0, sizeof(int), p->stream));
        return p->fail(SPADJ_ERR_TIMEOUT, "rb: a fused column stage gave up waiting for its operator block");
      }
      if (!std::isfinite(J_host[0])) return p->fail(SPADJ_ERR_NONFINITE, "rb: objective is not finite");
    }
    return SPADJ_OK;
  }

  spadj_status gradient(Problem* p, const double* x0, int n_steps, int objective_kind, const double* obj_data,
                        int ckpt_slots, double* J_host, double* grad, double* grad_p) override {
    (void)grad_p;
    if (objective_kind < 0) return p->fail(SPADJ_ERR_INVALID, "gradient: unknown objective");
    return reverse(p, x0, n_steps, ckpt_slots, objective_kind, obj_data, {}, nullptr, J_host, grad);
  }

  spadj_status vjp(Problem* p, const double* x0, int n_steps, int ckpt_slots, const std::vector<int>& seed_at,
                   const double* seeds, double* grad) override {
    return reverse(p, x0, n_steps, ckpt_slots, -1, nullptr, seed_at, seeds, nullptr, grad);
  }

  ~RB() override {
    for (cudaStream_t st : {gs, gs2, gsB, gsC})
      if (st) cudaStreamSynchronize(st);
    for (auto& os : opsets) {
      for (cudaGraphExec_t g : {os->gFwd[0], os->gFwd[1], os->gFwdB[0], os->gFwdB[1], os->gAdj[0][0], os->gAdj[0][1],
                                os->gAdj[1][0], os->gAdj[1][1], os->gStage[0], os->gStage[1], os->gAdjS[0][0],
                                os->gAdjS[0][1], os->gAdjS[1][0], os->gAdjS[1][1]})
        if (g) cudaGraphExecDestroy(g);
      os->phi.release();
      os->phiT.release();
    }
    for (cudaEvent_t e : {evIn, evOut, evFork, evJoin, evReady, evFree, evBdone, evAdj[0], evAdj[1], evCopied[0],
                          evCopied[1], evStaged[0], evStaged[1], evCdone})
      if (e) cudaEventDestroy(e);
    for (cudaStream_t st : {gs, gs2, gsB, gsC})
      if (st) cudaStreamDestroy(st);
    for (WS& l : ws) {
      for (DevBuf* b : {&l.Z, &l.Y, &l.G0, &l.G1, &l.f0, &l.f1, &l.x1}) b->release();
      for (int i = 0; i < 4; ++i)
        for (DevBuf* b : {&l.rx[i], &l.rv[i], &l.rf[i]}) b->release();
    }
    for (int i = 0; i < 4; ++i)
      for (DevBuf* b : {&tdx[i], &tdv[i], &tdf[i], &axb[i], &avb[i], &afb[i]}) b->release();
    for (DevBuf* b : {&aacc, &atmp, &axs}) b->release();
    errbuf.release();
    for (DevBuf* b : {&wm, &czE, &cdzE, &gzF, &gzTE, &czTF, &cdzTF, &gmat, &dG, &Gb, &Fg, &df0, &df1, &dx1,
                      &vb2, &vb1, &xb1, &tmpx, &tmpy, &ybar, &ybar2, &cur, &nxt, &curB, &nxtB, &partial, &Jdev,
                      &seedbuf, &slots, &traj_tmp})
      b->release();
    hslots.release();
  }
};

}  // namespace

spadj_status rb_set_dt_schedule(EqImpl* impl, Problem* p, int n, const double* dts) {
  RB* r = dynamic_cast<RB*>(impl);
  if (!r) return p->fail(SPADJ_ERR_UNSUPPORTED, "set_dt_schedule: only defined for the Rayleigh-Benard problem");
  return r->set_schedule(p, n, dts);
}

EqImpl* make_rb(Problem* p, spadj_status* st) {
  RB* r = new RB();
  *st = r->init(p);
  if (*st != SPADJ_OK) {
    delete r;
    return nullptr;
  }
  return r;
}

spadj_status rb_pencil_solve(EqImpl* impl, Problem* p, int transpose, const double* v, double* x) {
  RB* r = dynamic_cast<RB*>(impl);
  if (!r) return p->fail(SPADJ_ERR_UNSUPPORTED, "solve: only defined for the Rayleigh-Benard pencils");
  return r->pencil_solve(p, transpose, v, x);
}

int rb_last_recompute(EqImpl* impl) {
  RB* r = dynamic_cast<RB*>(impl);
  return r ? r->last_recompute : -1;
}

// ---- transform without allocation ----------------------------------------------------------
//
// Static device scratch for spadj_transform_noalloc: one mixed (z-grid x x-spectral) array of
// at most kNoAllocScratch complex entries (4 MiB).  Every GPU that loads the library holds it
// until the process exits.  Host code may not use the symbol as a device address; the
// address is fetched once per device with cudaGetSymbolAddress while that device is current.
constexpr size_t kNoAllocScratch = (size_t)1 << 18;
static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocScratch];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double2* g_noalloc_ptr[kMaxDevices] = {nullptr};
}  // namespace

spadj_status rb_transform_noalloc(EqImpl* impl, Problem* p, int kind, const double* in, double* out) {
  RB* r = dynamic_cast<RB*>(impl);
  if (!r) return p->fail(SPADJ_ERR_UNSUPPORTED, "transform_noalloc: only defined for the Rayleigh-Benard problem");
  if (kind < 0 || kind > 3) return p->fail(SPADJ_ERR_INVALID, "transform_noalloc: kind must be 0..3");
  const size_t need = (size_t)r->Mz * r->Kx;
  if (need > kNoAllocScratch)
    return p->fail(SPADJ_ERR_INVALID, "transform_noalloc: (3*n[1]/2) * (n[0]/2) = " + std::to_string(need) +
                                          " exceeds the static scratch of " + std::to_string(kNoAllocScratch) +
                                          " complex entries");
  int dev = 0;
  SPADJ_CUDA_TRY(p, cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return p->fail(SPADJ_ERR_INVALID, "transform_noalloc: device ordinal out of range");
  double2* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess)
        return p->fail(SPADJ_ERR_CUDA, std::string("transform_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_noalloc_ptr[dev] = static_cast<double2*>(ptr);
    }
    scratch = g_noalloc_ptr[dev];
  }
  return r->transform_into(p, kind, in, out, scratch);
}

}  // namespace spadj
