// Linear stability eigenvalues of plane shear flows and their adjoint-based parameter
// sensitivities for a batch of pencils (Problem types, "Eigenvalue problems"; Parametric
// sensitivity example).
//
// Pencil p has wavenumbers (alpha_p, beta_p), Reynolds number Re_p and a complex shift
// sigma_p.  The host factorises A_p = sigma_p M + L_p once (couette_setup.cpp, build_evp) and
// keeps T_p = A_p^-1 [S1S0 on the momentum rows] and RH_p = A_p^-H [e_0..e_{3N-1}] (the
// adjoint solve with the same factors).  The prognostic block Phi_p (first 3N rows of T_p)
// has eigenvalues mu = 1 / (sigma_p - lambda), so on the GPU:
//
//   1. shift-invert power iteration on Phi_p for the right eigenvector x and, in the same pass
//      over Phi_p, on Phi_p^H for the left eigenvector psi (the adjoint eigenproblem); the
//      two-sided Rayleigh quotient mu = psi^H Phi x / psi^H x gives lambda = sigma - 1/mu;
//   2. the full eigenvectors X = T_p x (velocity, pressure, tau variables) and
//      Y = RH_p psi, which solve (lambda M + L) X = 0 and (conj(lambda) M^H + L^H) Y = 0;
//   3. eq. eigenvalue_sens, dlambda/dp = -<Y, dL/dp X> / <Y, M X> for p = Re, alpha, beta
//      (M does not depend on them), with dL/dp applied from the N x N ultraspherical blocks.
#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "couette_setup.h"
#include "problem.h"
#include "rb_setup.h"

namespace spadj {
namespace {

constexpr int kEvpThreads = 256;
constexpr int kEvpWarps = kEvpThreads / 32;
constexpr int kEvpMaxChunks = 12;  // 3N <= 384: N <= 128
constexpr int kEvpOut = 10;        // lambda, dlambda/dRe, dlambda/dalpha, dlambda/dbeta, residuals

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum of NV values per thread (fixed warp-then-block order); every thread
// receives the totals.  red holds kEvpWarps * NV doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[warp * NV + i] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = 0.0;
    for (int w = 0; w < kEvpWarps; ++w) s += red[w * NV + i];
    v[i] = s;
  }
}

constexpr int kRows = 4;       // rows per warp block in evp_iter_kernel (2 kRows partial sums per lane)
constexpr int kRowsLog2V = 3;  // log2(2 kRows)

// Warp reduction of 2 kRows values per lane at once: a butterfly in which every exchange halves
// the values a lane carries (offsets 16, 8, ...; the lane keeps the half selected by that bit of
// its index) until one is left, then plain exchanges at the remaining offsets.  Every lane of the
// group l >> (5 - kRowsLog2V) = m ends with the total of value m.  2 kRows + 1 additions per lane
// for 2 kRows sums instead of 5 per sum; fixed order, so deterministic.
__device__ __forceinline__ double warp_reduce_rows(double (&v)[2 * kRows], int lane) {
  int off = 16;
#pragma unroll
  for (int half = kRows; half >= 1; half >>= 1, off >>= 1) {
    const bool hi = (lane & off) != 0;
#pragma unroll
    for (int j = 0; j < half; ++j) {
      const double send = hi ? v[j] : v[j + half];
      const double keep = hi ? v[j + half] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  double t = v[0];
#pragma unroll
  for (int o = 16 >> kRowsLog2V; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

struct EvpIterArgs {
  const double2* T;      // [P][nv][H]: rows 0..H-1 are Phi
  double2* x;            // [P][H] right iterate (in / out)
  double2* psi;          // [P][H] left iterate (in / out)
  const double* shift;   // [P][2]
  double* out;           // [P][kEvpOut]
  int H, nv, n_iter;
};

// One CTA per pencil: n_iter steps of x <- Phi x / |Phi x|, psi <- Phi^H psi / |Phi^H psi| with
// each row of Phi read once per step for both products (warps over rows, lanes over columns,
// coalesced), all in shared memory between steps.
// NC = ceil(3N / 32) column chunks per lane, fixed at compile time so that only the last chunk
// carries a bounds predicate.
template <int NC>
__global__ void __launch_bounds__(kEvpThreads, 2) evp_iter_kernel(const EvpIterArgs A) {
  const int p = blockIdx.x, H = A.H;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  extern __shared__ double2 evsm[];
  double2* x = evsm;
  double2* ps = x + H;
  double2* y = ps + H;
  double2* zp = y + H;                                    // [kEvpWarps][H] partial Phi^H psi
  double* red = reinterpret_cast<double*>(zp + (size_t)kEvpWarps * H);
  const double2* Tp = A.T + (size_t)p * A.nv * H;
  for (int k = threadIdx.x; k < H; k += blockDim.x) {
    x[k] = A.x[(size_t)p * H + k];
    ps[k] = A.psi[(size_t)p * H + k];
  }
  double mur = 0.0, mui = 0.0, res_r = 1.0, res_l = 1.0;
  for (int it = 0; it < A.n_iter; ++it) {
    __syncthreads();
    double2 zacc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) zacc[c] = make_double2(0.0, 0.0);
    // blocks of kRows rows per warp: each x chunk is read once per block, and the row sums of
    // the block are reduced together (warp_reduce_rows) instead of one butterfly per row
    for (int rb = warp * kRows; rb < H; rb += kRows * kEvpWarps) {
      double acc[2 * kRows];
      double2 pr[kRows];
#pragma unroll
      for (int i = 0; i < kRows; ++i) {
        acc[2 * i] = acc[2 * i + 1] = 0.0;
        pr[i] = rb + i < H ? ps[rb + i] : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int k = c * 32 + lane;
        if (c < NC - 1 || k < H) {
          const double2 xv = x[k];
#pragma unroll
          for (int i = 0; i < kRows; ++i) {
            if (rb + i >= H) continue;
            const double2 t = __ldg(&Tp[(size_t)(rb + i) * H + k]);
            acc[2 * i] = fma(t.x, xv.x, acc[2 * i]);
            acc[2 * i] = fma(-t.y, xv.y, acc[2 * i]);
            acc[2 * i + 1] = fma(t.x, xv.y, acc[2 * i + 1]);
            acc[2 * i + 1] = fma(t.y, xv.x, acc[2 * i + 1]);
            zacc[c].x = fma(t.x, pr[i].x, zacc[c].x);  // conj(t) * psi_r
            zacc[c].x = fma(t.y, pr[i].y, zacc[c].x);
            zacc[c].y = fma(t.x, pr[i].y, zacc[c].y);
            zacc[c].y = fma(-t.y, pr[i].x, zacc[c].y);
          }
        }
      }
      const double tot = warp_reduce_rows(acc, lane);
      // lane group m = lane >> (5 - kRowsLog2V) holds value m = 2 (row - rb) + component
      const int m = lane >> (5 - kRowsLog2V), r = rb + (m >> 1);
      if ((lane & ((1 << (5 - kRowsLog2V)) - 1)) == 0 && r < H) reinterpret_cast<double*>(y)[2 * r + (m & 1)] = tot;
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int k = c * 32 + lane;
      if (c < NC - 1 || k < H) zp[(size_t)warp * H + k] = zacc[c];
    }
    __syncthreads();
    // z = sum of the warp partials (into zp row 0); norms and the two-sided Rayleigh quotient
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < H; k += blockDim.x) {
      double2 z = zp[k];
      for (int w = 1; w < kEvpWarps; ++w) {
        const double2 q = zp[(size_t)w * H + k];
        z.x += q.x;
        z.y += q.y;
      }
      zp[k] = z;
      const double2 yk = y[k], xk = x[k], pk = ps[k];
      v[0] = fma(yk.x, yk.x, fma(yk.y, yk.y, v[0]));
      v[1] = fma(z.x, z.x, fma(z.y, z.y, v[1]));
      v[2] += pk.x * yk.x + pk.y * yk.y;  // psi^H y
      v[3] += pk.x * yk.y - pk.y * yk.x;
      v[4] += pk.x * xk.x + pk.y * xk.y;  // psi^H x
      v[5] += pk.x * xk.y - pk.y * xk.x;
    }
    block_sum<6>(v, red);
    const double dd = v[4] * v[4] + v[5] * v[5];
    if (dd > 0.0) {
      mur = (v[2] * v[4] + v[3] * v[5]) / dd;
      mui = (v[3] * v[4] - v[2] * v[5]) / dd;
    }
    if (it + 1 == A.n_iter) {  // residuals |Phi x - mu x| / |Phi x|, |Phi^H psi - conj(mu) psi| / |Phi^H psi|
      double r2[2] = {0.0, 0.0};
      for (int k = threadIdx.x; k < H; k += blockDim.x) {
        const double2 yk = y[k], xk = x[k], pk = ps[k], z = zp[k];
        const double ex = yk.x - (mur * xk.x - mui * xk.y), ey = yk.y - (mur * xk.y + mui * xk.x);
        const double fx = z.x - (mur * pk.x + mui * pk.y), fy = z.y - (mur * pk.y - mui * pk.x);
        r2[0] += ex * ex + ey * ey;
        r2[1] += fx * fx + fy * fy;
      }
      block_sum<2>(r2, red);
      res_r = v[0] > 0.0 ? sqrt(r2[0] / v[0]) : 1.0;
      res_l = v[1] > 0.0 ? sqrt(r2[1] / v[1]) : 1.0;
    }
    const double sy = v[0] > 0.0 ? 1.0 / sqrt(v[0]) : 0.0, sz = v[1] > 0.0 ? 1.0 / sqrt(v[1]) : 0.0;
    for (int k = threadIdx.x; k < H; k += blockDim.x) {
      const double2 yk = y[k], z = zp[k];
      x[k] = make_double2(yk.x * sy, yk.y * sy);
      ps[k] = make_double2(z.x * sz, z.y * sz);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < H; k += blockDim.x) {
    A.x[(size_t)p * H + k] = x[k];
    A.psi[(size_t)p * H + k] = ps[k];
  }
  if (threadIdx.x == 0) {
    double* o = A.out + (size_t)p * kEvpOut;
    const double m2 = mur * mur + mui * mui;
    // lambda = sigma - 1/mu
    o[0] = m2 > 0.0 ? A.shift[2 * p] - mur / m2 : 0.0;
    o[1] = m2 > 0.0 ? A.shift[2 * p + 1] + mui / m2 : 0.0;
    o[8] = res_r;
    o[9] = res_l;
  }
}

using EvpIterFn = void (*)(const EvpIterArgs);
const EvpIterFn kEvpIter[kEvpMaxChunks] = {
    evp_iter_kernel<1>, evp_iter_kernel<2>, evp_iter_kernel<3>, evp_iter_kernel<4>,
    evp_iter_kernel<5>, evp_iter_kernel<6>, evp_iter_kernel<7>, evp_iter_kernel<8>,
    evp_iter_kernel<9>, evp_iter_kernel<10>, evp_iter_kernel<11>, evp_iter_kernel<12>};

// X = T x and Y = RH psi (length nv each) for every pencil: warps over rows, lanes over columns.
__global__ void __launch_bounds__(kEvpThreads) evp_vectors_kernel(const double2* __restrict__ T,
                                                                  const double2* __restrict__ RH,
                                                                  const double2* __restrict__ x,
                                                                  const double2* __restrict__ psi, int H, int nv,
                                                                  double2* __restrict__ XY) {
  const int p = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double2* xp = x + (size_t)p * H;
  const double2* pp = psi + (size_t)p * H;
  for (int rr = warp; rr < 2 * nv; rr += kEvpWarps) {
    const int which = rr / nv, r = rr - which * nv;
    const double2* row = (which == 0 ? T : RH) + ((size_t)p * nv + r) * H;
    const double2* v = which == 0 ? xp : pp;
    double ax = 0.0, ay = 0.0;
    for (int k = lane; k < H; k += 32) {
      const double2 t = __ldg(&row[k]), q = __ldg(&v[k]);
      ax = fma(t.x, q.x, ax);
      ax = fma(-t.y, q.y, ax);
      ay = fma(t.x, q.y, ay);
      ay = fma(t.y, q.x, ay);
    }
    ax = warp_sum(ax);
    ay = warp_sum(ay);
    if (lane == 0) XY[((size_t)p * 2 + which) * nv + r] = make_double2(ax, ay);
  }
}

struct EvpSensArgs {
  const double2* XY;                 // [P][2][nv]: X, Y
  const double* prm;                 // [P][3]: alpha, beta, Re
  const double *SS, *DD, *Um, *S0;   // N x N row-major
  double* out;                       // [P][kEvpOut]
  int N, nv, lift_row;
  double lift_val;
};

// eq. eigenvalue_sens for p = Re, alpha, beta.  With lap = DD - k^2 SS on each velocity block:
//   dL/dRe    = lap / Re^2 on the u, v, w blocks, lift_val / Re^2 at the tau_q1 lifts;
//   dL/dalpha = 2 alpha nu SS + i Umat on the blocks, i SS at (u-eq, p), i S0 at (cont, u);
//   dL/dbeta  = 2 beta nu SS on the blocks, i SS at (v-eq, p), i S0 at (cont, v);
// <Y, M X> = sum over u, v, w of Y_q^H SS X_q.
__global__ void __launch_bounds__(kEvpThreads) evp_sens_kernel(const EvpSensArgs A) {
  const int p = blockIdx.x, N = A.N, nv = A.nv;
  extern __shared__ double2 essm[];
  double2* X = essm;
  double2* Y = X + nv;
  double* red = reinterpret_cast<double*>(Y + nv);
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    X[i] = A.XY[((size_t)p * 2 + 0) * nv + i];
    Y[i] = A.XY[((size_t)p * 2 + 1) * nv + i];
  }
  __syncthreads();
  const double al = A.prm[3 * p], be = A.prm[3 * p + 1], Re = A.prm[3 * p + 2];
  const double nu = 1.0 / Re, k2 = al * al + be * be;
  // accumulators (re, im): den, nRe, nA, nB
  double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  auto cjmul_add = [](double* acc, double2 y, double2 z) {  // acc += conj(y) z
    acc[0] += y.x * z.x + y.y * z.y;
    acc[1] += y.x * z.y - y.y * z.x;
  };
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double2 s[3], d[3], u[3], sp, s0u, s0v;
    for (int q = 0; q < 3; ++q) s[q] = d[q] = u[q] = make_double2(0.0, 0.0);
    sp = s0u = s0v = make_double2(0.0, 0.0);
    for (int j = 0; j < N; ++j) {
      const double ss = __ldg(&A.SS[(size_t)i * N + j]), dd = __ldg(&A.DD[(size_t)i * N + j]);
      const double um = __ldg(&A.Um[(size_t)i * N + j]), s0 = __ldg(&A.S0[(size_t)i * N + j]);
      for (int q = 0; q < 3; ++q) {
        const double2 xq = X[q * N + j];
        s[q].x = fma(ss, xq.x, s[q].x); s[q].y = fma(ss, xq.y, s[q].y);
        d[q].x = fma(dd, xq.x, d[q].x); d[q].y = fma(dd, xq.y, d[q].y);
        u[q].x = fma(um, xq.x, u[q].x); u[q].y = fma(um, xq.y, u[q].y);
      }
      const double2 xp = X[3 * N + j], xu = X[j], xv = X[N + j];
      sp.x = fma(ss, xp.x, sp.x); sp.y = fma(ss, xp.y, sp.y);
      s0u.x = fma(s0, xu.x, s0u.x); s0u.y = fma(s0, xu.y, s0u.y);
      s0v.x = fma(s0, xv.x, s0v.x); s0v.y = fma(s0, xv.y, s0v.y);
    }
    for (int q = 0; q < 3; ++q) {
      const double2 yq = Y[q * N + i];
      cjmul_add(&v[0], yq, s[q]);
      cjmul_add(&v[2], yq, make_double2(d[q].x - k2 * s[q].x, d[q].y - k2 * s[q].y));
      // 2 alpha nu s + i u
      cjmul_add(&v[4], yq, make_double2(2.0 * al * nu * s[q].x - u[q].y, 2.0 * al * nu * s[q].y + u[q].x));
      cjmul_add(&v[6], yq, make_double2(2.0 * be * nu * s[q].x, 2.0 * be * nu * s[q].y));
    }
    const double2 yu = Y[i], yv = Y[N + i], yp = Y[3 * N + i];
    cjmul_add(&v[4], yu, make_double2(-sp.y, sp.x));    // i SS p in the u-equation
    cjmul_add(&v[4], yp, make_double2(-s0u.y, s0u.x));  // i S0 u in continuity
    cjmul_add(&v[6], yv, make_double2(-sp.y, sp.x));
    cjmul_add(&v[6], yp, make_double2(-s0v.y, s0v.x));
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) {  // tau_q1 lift entries of -nu d/dz(lift)
      const double2 xt = X[4 * N + 2 * q];
      cjmul_add(&v[2], Y[q * N + A.lift_row], make_double2(A.lift_val * xt.x, A.lift_val * xt.y));
    }
  block_sum<8>(v, red);
  if (threadIdx.x == 0) {
    double* o = A.out + (size_t)p * kEvpOut;
    const double dr = v[0], di = v[1], dd = dr * dr + di * di;
    const double sc[3] = {1.0 / (Re * Re), 1.0, 1.0};
    for (int t = 0; t < 3; ++t) {
      const double nr = sc[t] * v[2 + 2 * t], ni = sc[t] * v[3 + 2 * t];
      // -num / den
      o[2 + 2 * t] = dd > 0.0 ? -(nr * dr + ni * di) / dd : 0.0;
      o[3 + 2 * t] = dd > 0.0 ? -(ni * dr - nr * di) / dd : 0.0;
    }
  }
}

struct ShearEvp : EqImpl {
  int N = 0, H = 0, nv = 0, base = 0, Pmax = 0;
  rbhost::Operators ops;
  DevBuf T, RH, XY, shiftd, prmd, mats;

  size_t state_len(int which) const override { return which == 0 ? (size_t)Pmax * H * 2 : 0; }

  spadj_status init(Problem* p) {
    const spadj_desc& d = p->desc;
    N = d.n[2];
    base = (int)d.params[0];
    Pmax = d.batch;
    if (N < 8 || 3 * N > 32 * kEvpMaxChunks)
      return p->fail(SPADJ_ERR_INVALID, "shear evp: need 8 <= n[2] <= " + std::to_string(32 * kEvpMaxChunks / 3));
    if ((base != 0 && base != 1) || (double)base != d.params[0])
      return p->fail(SPADJ_ERR_INVALID, "shear evp: params[0] must be 0 (plane Couette) or 1 (plane Poiseuille)");
    H = 3 * N;
    nv = 4 * N + 7;
    ops = rbhost::build_operators(N, 3 * N / 2, 1.0);
    std::vector<double> Um, UP;
    couhost::base_flow(ops, base, Um, UP);
    std::vector<double> m;
    m.insert(m.end(), ops.SS.begin(), ops.SS.end());
    m.insert(m.end(), ops.DD.begin(), ops.DD.end());
    m.insert(m.end(), Um.begin(), Um.end());
    m.insert(m.end(), ops.S0.begin(), ops.S0.end());
    SPADJ_CUDA_TRY(p, mats.ensure(sizeof(double) * m.size()));
    SPADJ_CUDA_TRY(p, cudaMemcpy(mats.ptr, m.data(), sizeof(double) * m.size(), cudaMemcpyHostToDevice));
    const size_t ismem = sizeof(double2) * (size_t)(3 + kEvpWarps) * H + sizeof(double) * kEvpWarps * 6;
    if (ismem > 48 * 1024)
      SPADJ_CUDA_TRY(p, cudaFuncSetAttribute(kEvpIter[(H + 31) / 32 - 1],
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem));
    return SPADJ_OK;
  }

  spadj_status eigen(Problem* p, int P, const double* prm, const double* shift, int n_iter, double* x, double* psi,
                     double* out) {
    if (P < 1 || P > Pmax) return p->fail(SPADJ_ERR_INVALID, "eigen: n_pencils must be in 1..batch");
    if (n_iter < 1) return p->fail(SPADJ_ERR_INVALID, "eigen: n_iter < 1");
    for (int i = 0; i < P; ++i)
      if (!(prm[3 * i + 2] > 0.0) || !std::isfinite(prm[3 * i]) || !std::isfinite(prm[3 * i + 1]))
        return p->fail(SPADJ_ERR_INVALID, "eigen: need finite wavenumbers and Re > 0");
    std::vector<double> th, rh;
    std::string err;
    if (!couhost::build_evp(ops, base, P, prm, shift, th, rh, &err)) return p->fail(SPADJ_ERR_INVALID, err);
    SPADJ_CUDA_TRY(p, T.ensure(sizeof(double) * th.size()));
    SPADJ_CUDA_TRY(p, RH.ensure(sizeof(double) * rh.size()));
    SPADJ_CUDA_TRY(p, XY.ensure(sizeof(double2) * (size_t)P * 2 * nv));
    SPADJ_CUDA_TRY(p, shiftd.ensure(sizeof(double) * 2 * P));
    SPADJ_CUDA_TRY(p, prmd.ensure(sizeof(double) * 3 * P));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(T.ptr, th.data(), sizeof(double) * th.size(), cudaMemcpyHostToDevice, p->stream));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(RH.ptr, rh.data(), sizeof(double) * rh.size(), cudaMemcpyHostToDevice, p->stream));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(shiftd.ptr, shift, sizeof(double) * 2 * P, cudaMemcpyHostToDevice, p->stream));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(prmd.ptr, prm, sizeof(double) * 3 * P, cudaMemcpyHostToDevice, p->stream));
    EvpIterArgs ia{};
    ia.T = T.as<double2>();
    ia.x = reinterpret_cast<double2*>(x);
    ia.psi = reinterpret_cast<double2*>(psi);
    ia.shift = shiftd.as<double>();
    ia.out = out;
    ia.H = H;
    ia.nv = nv;
    ia.n_iter = n_iter;
    const size_t ismem = sizeof(double2) * (size_t)(3 + kEvpWarps) * H + sizeof(double) * kEvpWarps * 6;
    cudaEvent_t t0 = p->tic();
    kEvpIter[(H + 31) / 32 - 1]<<<P, kEvpThreads, ismem, p->stream>>>(ia);
    // two complex matvecs per step over the 3N x 3N block: 16 flops per entry
    p->toc(t0, KC_SOLVE, 16.0 * (double)H * H * P * n_iter);
    spadj_status s = check_launch(p, "evp iterate");
    if (s != SPADJ_OK) return s;
    cudaEvent_t t1 = p->tic();
    evp_vectors_kernel<<<P, kEvpThreads, 0, p->stream>>>(T.as<double2>(), RH.as<double2>(), ia.x, ia.psi, H, nv,
                                                         XY.as<double2>());
    p->toc(t1, KC_OBJECTIVE, 16.0 * (double)nv * H * P);
    if ((s = check_launch(p, "evp vectors")) != SPADJ_OK) return s;
    EvpSensArgs sa{};
    sa.XY = XY.as<double2>();
    sa.prm = prmd.as<double>();
    const size_t nn = (size_t)N * N;
    sa.SS = mats.as<double>();
    sa.DD = sa.SS + nn;
    sa.Um = sa.DD + nn;
    sa.S0 = sa.Um + nn;
    sa.out = out;
    sa.N = N;
    sa.nv = nv;
    sa.lift_row = ops.lift_row;
    sa.lift_val = ops.lift_val;
    const size_t ssmem = sizeof(double2) * 2 * nv + sizeof(double) * kEvpWarps * 8;
    cudaEvent_t t2 = p->tic();
    evp_sens_kernel<<<P, kEvpThreads, ssmem, p->stream>>>(sa);
    p->toc(t2, KC_OBJECTIVE, (12.0 * 4.0 * N * N + 64.0 * N) * P);
    if ((s = check_launch(p, "evp sensitivity")) != SPADJ_OK) return s;
    // the host operator buffers must outlive the asynchronous copies
    SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    return SPADJ_OK;
  }

  // ---- operations of the time-dependent problems are not defined here ------------------------
  spadj_status unsupported(Problem* p, const char* what) {
    return p->fail(SPADJ_ERR_UNSUPPORTED, std::string(what) + ": not defined for the shear-flow eigenproblem");
  }
  spadj_status transform(Problem* p, int, const double*, double*) override { return unsupported(p, "transform"); }
  spadj_status eval_F(Problem* p, int, const double*, const double*, double*) override {
    return unsupported(p, "eval_F");
  }
  spadj_status forward(Problem* p, int, const double*, double*, double*) override { return unsupported(p, "forward"); }
  spadj_status tangent(Problem* p, int, const double*, const double*, double*) override {
    return unsupported(p, "tangent");
  }
  spadj_status adjoint(Problem* p, int, const double*, const double*, double*, double*) override {
    return unsupported(p, "adjoint");
  }
  spadj_status objective(Problem* p, int, const double*, const double*, double*, double*) override {
    return unsupported(p, "objective");
  }
  spadj_status gradient(Problem* p, const double*, int, int, const double*, int, double*, double*, double*) override {
    return unsupported(p, "gradient");
  }
  spadj_status vjp(Problem* p, const double*, int, int, const std::vector<int>&, const double*, double*) override {
    return unsupported(p, "vjp");
  }
};

}  // namespace

EqImpl* make_shear_evp(Problem* p, spadj_status* st) {
  ShearEvp* e = new ShearEvp();
  *st = e->init(p);
  if (*st != SPADJ_OK) {
    delete e;
    return nullptr;
  }
  return e;
}

spadj_status evp_eigen(EqImpl* impl, Problem* p, int P, const double* prm, const double* shift, int n_iter, double* x,
                       double* psi, double* out) {
  ShearEvp* e = dynamic_cast<ShearEvp*>(impl);
  if (!e) return p->fail(SPADJ_ERR_UNSUPPORTED, "eigen: only defined for the shear-flow eigenproblem");
  return e->eigen(p, P, prm, shift, n_iter, x, psi, out);
}

}  // namespace spadj
