// Device kernels of the Rayleigh-Benard path (Fourier x x Chebyshev z, FP64).
//
// Layouts (Kx = Nx/2 x-modes, N Chebyshev modes, Mx x Mz dealiased grid):
//   coefficients  [field][Kx][N]   complex (one pencil contiguous)
//   mixed         [Mz][Kx]         complex (z on the grid, x in spectral space)
//   grid          [Mz][Mx]         real
// The z transforms are small dense real matrices applied to complex columns; they use
// the reflection symmetry of the Gauss grid (xi_{Mz-1-j} = -xi_j, T_n(-xi) = (-1)^n T_n(xi))
// so every output pair (j, Mz-1-j) costs one half-length dot product ("expand"), and
// every grid-to-coefficient reduction runs over Mz/2 folded samples ("fold").
#pragma once
#include <algorithm>
#include <cooperative_groups.h>

#include "fft.cuh"
#include "pdl.cuh"

namespace spadj {
namespace rbk {
// internal linkage: every translation unit that includes this header gets its own kernels
namespace {

constexpr int kZMaxJobs = 9;
constexpr int kXMaxJobs = 12;

// One z-transform job: out = sum_t alpha_t * mat_t * v_t (+ sum_a beta_a * add_a), where the
// staged column v_t = mult_t(in_t) + sum_{e: xterm_e = t} xalpha_e * xmult_e(xin_e) combines
// inputs that share matrix t before the matrix is applied (in_t may be NULL; mult: 0 none,
// 1 i*kx, 2 i*ky of the column; only the Fourier-Fourier-Chebyshev layouts use them).
//   expand: K = N coefficients -> I = Mz grid rows; mat_t is (Mz/2) x N (rows j < Mz/2)
//   fold:   K = Mz grid rows -> I = N coefficients; mat_t is N x (Mz/2) (columns j < Mz/2)
// deriv_t = 1 when mat_t has the reflection parity of a z-derivative (-(-1)^n).
struct ZJob {
  const double2* in[2];
  const double* mat[2];
  double alpha[2];
  int deriv[2];
  int mult[2];
  int nterm;
  const double2* xin[2];
  double xalpha[2];
  int xmult[2];
  int xterm[2];
  int nx;
  const double2* add[3];
  double beta[3];
  int nadd;
  double2* out;
  int I, K;
  int ik, im;  // in(k, m) = in[k*ik + m*im]
  int oi, om;  // out(i, m) = out[i*oi + m*om]
};
struct ZJobs {
  ZJob j[kZMaxJobs];
  int n;
  int ncols;  // columns (pencils)
  int expand; // 1: expand, 0: fold
  // column m = jy * kxn + mx has wavenumbers kx = kxs * mx, ky = kys * (jy < nyk/2 ? jy : jy - nyk)
  int kxn, nyk;
  double kxs, kys;
};

// i * (kx or ky of column m) * v
__device__ __forceinline__ double2 zmult(const ZJobs& js, int type, int m, double2 v) {
  if (type == 0) return v;
  double k;
  if (type == 1) {
    k = js.kxs * (m % js.kxn);
  } else {
    const int jy = m / js.kxn;
    k = js.kys * (jy < js.nyk / 2 ? jy : jy - js.nyk);
  }
  return make_double2(-k * v.y, k * v.x);
}

// One CTA per (column, job); the reduction of every output is split over the two lanes of a
// lane pair and combined with a shuffle, so an expand job runs 2*Mz/2 threads and a fold job
// 2*N threads per column.
constexpr int kTM = 1;  // columns per CTA

__host__ __device__ inline int zmm_threads(int expand, int I) { return 2 * (expand ? I / 2 : I); }

__global__ void __launch_bounds__(256) zmm_kernel(const __grid_constant__ ZJobs js) {
  pdl_trigger();
  pdl_wait();
  const ZJob& J = js.j[blockIdx.y];
  const int m = blockIdx.x;
  extern __shared__ double2 sb[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int K = J.K, I = J.I;
  const int Kh = js.expand ? K : K / 2;  // staged entries per term (and per s/d array)
  // stage this column: expand -> coefficients; fold -> (s, d) = f_j +- f_{Mz-1-j}
  auto comb = [&](int t, int k) {
    double2 v = J.in[t] ? zmult(js, J.mult[t], m, J.in[t][(size_t)m * J.im + (size_t)k * J.ik])
                        : make_double2(0.0, 0.0);
    for (int e = 0; e < J.nx; ++e) {
      if (J.xterm[e] != t) continue;
      const double2 x = zmult(js, J.xmult[e], m, J.xin[e][(size_t)m * J.im + (size_t)k * J.ik]);
      v.x = fma(J.xalpha[e], x.x, v.x);
      v.y = fma(J.xalpha[e], x.y, v.y);
    }
    return v;
  };
  for (int t = 0; t < J.nterm; ++t) {
    double2* s = sb + (size_t)t * 2 * Kh;
    for (int k = tid; k < Kh; k += nt) {
      const double2 v = comb(t, k);
      if (js.expand) {
        s[k] = v;
      } else {
        const double2 v2 = comb(t, K - 1 - k);
        s[k] = make_double2(v.x + v2.x, v.y + v2.y);       // s_j
        s[Kh + k] = make_double2(v.x - v2.x, v.y - v2.y);  // d_j
      }
    }
  }
  __syncthreads();
  const int u = tid >> 1, hf = tid & 1;
  if (js.expand) {
    const int Ih = I / 2;
    if (u >= Ih) return;
    const int k0 = hf * (K / 2), k1 = hf ? K : K / 2;  // K even: both halves start on an even k
    double2 lo = make_double2(0.0, 0.0), hi = make_double2(0.0, 0.0);
    for (int t = 0; t < J.nterm; ++t) {
      const double* a = J.mat[t] + (size_t)u * K;
      const double2* s = sb + (size_t)t * 2 * Kh;
      double2 E = make_double2(0.0, 0.0), O = make_double2(0.0, 0.0);
#pragma unroll 4
      for (int k = k0; k < k1; k += 2) {
        const double ae = __ldg(a + k), ao = __ldg(a + k + 1);
        const double2 ve = s[k], vo = s[k + 1];
        E.x = fma(ae, ve.x, E.x); E.y = fma(ae, ve.y, E.y);
        O.x = fma(ao, vo.x, O.x); O.y = fma(ao, vo.y, O.y);
      }
      E.x += __shfl_xor_sync(__activemask(), E.x, 1);
      E.y += __shfl_xor_sync(__activemask(), E.y, 1);
      O.x += __shfl_xor_sync(__activemask(), O.x, 1);
      O.y += __shfl_xor_sync(__activemask(), O.y, 1);
      const double al = J.alpha[t];
      // out_j = E + O ; out_{Mz-1-j} = E - O (parity (-1)^n) or -E + O (derivative parity)
      const double se = J.deriv[t] ? -1.0 : 1.0;
      lo.x = fma(al, E.x + O.x, lo.x); lo.y = fma(al, E.y + O.y, lo.y);
      hi.x = fma(al, se * (E.x - O.x), hi.x); hi.y = fma(al, se * (E.y - O.y), hi.y);
    }
    if (hf == 0) {
      const size_t o1 = (size_t)u * J.oi + (size_t)m * J.om;
      const size_t o2 = (size_t)(I - 1 - u) * J.oi + (size_t)m * J.om;
      for (int a = 0; a < J.nadd; ++a) {
        const double2 p = J.add[a][o1], q = J.add[a][o2];
        lo.x = fma(J.beta[a], p.x, lo.x); lo.y = fma(J.beta[a], p.y, lo.y);
        hi.x = fma(J.beta[a], q.x, hi.x); hi.y = fma(J.beta[a], q.y, hi.y);
      }
      J.out[o1] = lo;
      J.out[o2] = hi;
    }
  } else {
    if (u >= I) return;
    const int Kf = K / 2;
    const int k0 = hf * (Kf / 2), k1 = hf ? Kf : Kf / 2;
    double2 acc = make_double2(0.0, 0.0);
    for (int t = 0; t < J.nterm; ++t) {
      const double* a = J.mat[t] + (size_t)u * Kf;
      // even rows pair with s for parity (-1)^n, with d for derivative parity
      const bool use_s = ((u & 1) == 0) != (J.deriv[t] != 0);
      const double2* s = sb + (size_t)t * 2 * Kh + (use_s ? 0 : Kh);
      double2 v0 = make_double2(0.0, 0.0), v1 = make_double2(0.0, 0.0);
      int k = k0;
#pragma unroll 4
      for (; k + 1 < k1; k += 2) {
        const double a0 = __ldg(a + k), a1 = __ldg(a + k + 1);
        const double2 x0 = s[k], x1 = s[k + 1];
        v0.x = fma(a0, x0.x, v0.x); v0.y = fma(a0, x0.y, v0.y);
        v1.x = fma(a1, x1.x, v1.x); v1.y = fma(a1, x1.y, v1.y);
      }
      if (k < k1) {
        const double a0 = __ldg(a + k);
        const double2 x0 = s[k];
        v0.x = fma(a0, x0.x, v0.x); v0.y = fma(a0, x0.y, v0.y);
      }
      double vx = v0.x + v1.x, vy = v0.y + v1.y;
      vx += __shfl_xor_sync(__activemask(), vx, 1);
      vy += __shfl_xor_sync(__activemask(), vy, 1);
      acc.x = fma(J.alpha[t], vx, acc.x); acc.y = fma(J.alpha[t], vy, acc.y);
    }
    if (hf == 0) {
      const size_t o = (size_t)u * J.oi + (size_t)m * J.om;
      for (int a = 0; a < J.nadd; ++a) {
        const double2 p = J.add[a][o];
        acc.x = fma(J.beta[a], p.x, acc.x); acc.y = fma(J.beta[a], p.y, acc.y);
      }
      J.out[o] = acc;
    }
  }
}

// One x-transform job over all Mz rows.
//   dir 0 (c2r): grid row j = sum over the Hermitian spectrum of mult(k) * cin[j][k]
//                with weights (w0 on k = 0, w on k >= 1), mult = 1 or i*k.
//   dir 1 (r2c): cout[j][k] = sum_t mult_t(k) * scale(k) * FFT(rin_t row j)[k], k < Kx,
//                mult = 1 or -i*k, scale = s0 (k = 0) or s (k >= 1).
struct XJob {
  int dir;
  // dir 1 with nprod > 0: the input row is the grid product sum_t ps_t G[pa_t] G[pb_t] of
  // grid fields (slots of G, npts points each), or its tangent
  // sum_t ps_t (dG[pa_t] G[pb_t] + G[pa_t] dG[pb_t]) when dG is non-null
  int nprod;
  int pa[2], pb[2];
  double ps[2];
  const double* G;
  const double* dG;
  int npts;
  const double2* cin;
  int cmul;
  double w0, w;
  double* rout;
  const double* rin[2];
  int rmul[2];
  int nr;
  double s0, s;
  double2* cout;
};
struct XJobs {
  XJob j[kXMaxJobs];
  int n;
};

struct XParams {
  int Kx, Mx, L;
  double kscale;
  FFTPlan plan;
  const double2* WM;
};

__global__ void __launch_bounds__(64) xfft_kernel(const __grid_constant__ XJobs js, XParams P) {
  pdl_trigger();
  pdl_wait();
  const XJob& J = js.j[blockIdx.y];
  const int row = blockIdx.x;
  const int L = P.L, Kx = P.Kx, Mx = P.Mx;
  extern __shared__ double2 sx[];
  double2* A = sx;
  double2* B = A + L;
  double2* C = B + L;
  double2* D = C + L;
  double2* S = D + L;  // Kx
  if (J.dir == 0) {
    const double2* src = J.cin + (size_t)row * Kx;
    for (int k = threadIdx.x; k < Kx; k += blockDim.x) {
      double2 v = src[k];
      if (J.cmul == 1) {  // i k v
        const double kk = P.kscale * k;
        v = make_double2(-kk * v.y, kk * v.x);
      }
      S[k] = v;
    }
    __syncthreads();
    c2r_pre(A, [&](int k) { return S[k]; }, Kx, L, P.WM, J.w0, J.w);
    __syncthreads();
    double2* z = cfft_smem(A, B, P.plan, P.WM, +1);
    double2* g = reinterpret_cast<double2*>(J.rout + (size_t)row * Mx);
    for (int j = threadIdx.x; j < L; j += blockDim.x) g[j] = z[j];
  } else {
    if (J.nprod > 0) {
      auto rowp = [&](const double* base, int slot) {
        return reinterpret_cast<const double2*>(base + (size_t)slot * J.npts + (size_t)row * Mx);
      };
      const double2 *a0 = rowp(J.G, J.pa[0]), *b0 = rowp(J.G, J.pb[0]);
      const double2 *a1 = rowp(J.G, J.pa[1]), *b1 = rowp(J.G, J.pb[1]);
      const double p0 = J.ps[0], p1 = J.ps[1];
      if (!J.dG) {
        for (int j = threadIdx.x; j < L; j += blockDim.x) {
          const double2 a = a0[j], b = b0[j], c = a1[j], d = b1[j];
          A[j] = make_double2(fma(p0 * a.x, b.x, p1 * (c.x * d.x)), fma(p0 * a.y, b.y, p1 * (c.y * d.y)));
        }
      } else {
        const double2 *da0 = rowp(J.dG, J.pa[0]), *db0 = rowp(J.dG, J.pb[0]);
        const double2 *da1 = rowp(J.dG, J.pa[1]), *db1 = rowp(J.dG, J.pb[1]);
        for (int j = threadIdx.x; j < L; j += blockDim.x) {
          const double2 a = a0[j], b = b0[j], c = a1[j], d = b1[j];
          const double2 da = da0[j], db = db0[j], dc = da1[j], dd = db1[j];
          A[j] = make_double2(p0 * (da.x * b.x + a.x * db.x) + p1 * (dc.x * d.x + c.x * dd.x),
                              p0 * (da.y * b.y + a.y * db.y) + p1 * (dc.y * d.y + c.y * dd.y));
        }
      }
    } else {
      for (int t = 0; t < J.nr; ++t) {
        double2* a = (t == 0) ? A : C;
        const double2* g = reinterpret_cast<const double2*>(J.rin[t] + (size_t)row * Mx);
        for (int j = threadIdx.x; j < L; j += blockDim.x) a[j] = g[j];
      }
    }
    __syncthreads();
    double2 *z0, *z1 = nullptr;
    if (J.nr > 1) {  // both inputs' transforms in the same passes (A|B and C|D are 2L apart)
      cfft_smem_sets<-1>(A, B, 2 * L, 2, P.plan, 1);
      z0 = (P.plan.nrad & 1) ? B : A;
      z1 = (P.plan.nrad & 1) ? D : C;
    } else {
      z0 = cfft_smem(A, B, P.plan, P.WM, -1);
    }
    double2* dst = J.cout + (size_t)row * Kx;
    // r2c post-processing for each input, combined
    for (int k = threadIdx.x; k < Kx; k += blockDim.x) {
      double2 acc = make_double2(0.0, 0.0);
      for (int t = 0; t < J.nr; ++t) {
        const double2* Z = (t == 0) ? z0 : z1;
        double2 X = r2c_combine2(Z[k], cconj(Z[k == 0 ? 0 : L - k]), __ldg(&P.WM[k]));  // twice the entry
        if (J.rmul[t] == 2) {  // -i k X
          const double kk = P.kscale * k;
          X = make_double2(kk * X.y, -kk * X.x);
        }
        acc = t == 0 ? X : cadd(acc, X);
      }
      const double sc = 0.5 * ((k == 0) ? J.s0 : J.s);
      double2 r = cscale(acc, sc);
      if (k == 0) r.y = 0.0;
      dst[k] = r;
    }
  }
}

constexpr int kXThreadsMax = 192;
// xfft_kernel's jobs for nb rows per CTA (nb <= 4): the rows are interleaved in shared memory
// (element e of row c at e * nb + c) and transformed together by cfft_smem_batch, so short rows
// keep all threads of the CTA busy in every Stockham pass and share its barriers.
__global__ void __launch_bounds__(kXThreadsMax) xfftm_kernel(const __grid_constant__ XJobs js, XParams P, int nb, int nrows) {
  pdl_trigger();
  pdl_wait();
  const XJob& J = js.j[blockIdx.y];
  const int row0 = blockIdx.x * nb;
  const int L = P.L, Kx = P.Kx, Mx = P.Mx;
  extern __shared__ double2 sx[];
  double2* A = sx;
  double2* B = A + (size_t)L * nb;
  double2* C = B + (size_t)L * nb;
  double2* D = C + (size_t)L * nb;
  double2* S = D + (size_t)L * nb;  // [nb][Kx]
  const int tid = threadIdx.x, nt = blockDim.x;
  if (J.dir == 0) {
    for (int idx = tid; idx < nb * Kx; idx += nt) {
      const int c = idx / Kx, k = idx - c * Kx;
      double2 v = make_double2(0.0, 0.0);
      if (row0 + c < nrows) {
        v = J.cin[(size_t)(row0 + c) * Kx + k];
        if (J.cmul == 1) {  // i k v
          const double kk = P.kscale * k;
          v = make_double2(-kk * v.y, kk * v.x);
        }
      }
      S[idx] = v;
    }
    __syncthreads();
    // packed spectrum of each real row (c2r_pre), interleaved
    for (int idx = tid; idx < nb * L; idx += nt) {
      const int k = idx / nb, c = idx - k * nb;
      const double2* Sr = S + (size_t)c * Kx;
      double2 xk = make_double2(0.0, 0.0), xc = make_double2(0.0, 0.0);
      if (k == 0) xk = make_double2(J.w0 * Sr[0].x, 0.0);
      else if (k < Kx) xk = cscale(Sr[k], J.w);
      const int kc = L - k;
      if (k > 0 && kc < Kx) xc = cconj(cscale(Sr[kc], J.w));
      A[idx] = c2r_combine(cadd(xk, xc), csub(xk, xc), __ldg(&P.WM[k]));
    }
    __syncthreads();
    const double2* z = cfft_smem_batch<1>(A, B, P.plan, P.WM, nb);
    for (int idx = tid; idx < nb * L; idx += nt) {
      const int c = idx / L, j = idx - c * L;
      if (row0 + c < nrows) reinterpret_cast<double2*>(J.rout + (size_t)(row0 + c) * Mx)[j] = z[j * nb + c];
    }
    return;
  }
  const int nin = J.nprod > 0 ? 1 : J.nr;
  for (int idx = tid; idx < nb * L; idx += nt) {
    const int c = idx / L, j = idx - c * L;
    double2 v0 = make_double2(0.0, 0.0), v1 = make_double2(0.0, 0.0);
    if (row0 + c < nrows) {
      const size_t ro = (size_t)(row0 + c) * Mx;
      if (J.nprod > 0) {
        auto at = [&](const double* base, int slot) {
          return reinterpret_cast<const double2*>(base + (size_t)slot * J.npts + ro)[j];
        };
        const double2 a = at(J.G, J.pa[0]), b = at(J.G, J.pb[0]), cc = at(J.G, J.pa[1]), d = at(J.G, J.pb[1]);
        const double p0 = J.ps[0], p1 = J.ps[1];
        if (!J.dG) {
          v0 = make_double2(fma(p0 * a.x, b.x, p1 * (cc.x * d.x)), fma(p0 * a.y, b.y, p1 * (cc.y * d.y)));
        } else {
          const double2 da = at(J.dG, J.pa[0]), db = at(J.dG, J.pb[0]), dc = at(J.dG, J.pa[1]), dd = at(J.dG, J.pb[1]);
          v0 = make_double2(p0 * (da.x * b.x + a.x * db.x) + p1 * (dc.x * d.x + cc.x * dd.x),
                            p0 * (da.y * b.y + a.y * db.y) + p1 * (dc.y * d.y + cc.y * dd.y));
        }
      } else {
        v0 = reinterpret_cast<const double2*>(J.rin[0] + ro)[j];
        if (nin > 1) v1 = reinterpret_cast<const double2*>(J.rin[1] + ro)[j];
      }
    }
    A[j * nb + c] = v0;
    if (nin > 1) C[j * nb + c] = v1;
  }
  __syncthreads();
  cfft_smem_sets<-1>(A, B, 2 * L * nb, nin, P.plan, nb);  // A|B and C|D are 2 L nb apart
  const double2* z0 = (P.plan.nrad & 1) ? B : A;
  const double2* z1 = (P.plan.nrad & 1) ? D : C;
  for (int idx = tid; idx < nb * Kx; idx += nt) {
    const int c = idx / Kx, k = idx - c * Kx;
    if (row0 + c >= nrows) continue;
    double2 acc = make_double2(0.0, 0.0);
    for (int t = 0; t < nin; ++t) {
      const double2* Z = t == 0 ? z0 : z1;
      double2 X = r2c_combine2(Z[k * nb + c], cconj(Z[(k == 0 ? 0 : L - k) * nb + c]), __ldg(&P.WM[k]));
      if (J.rmul[t] == 2) {  // -i k X
        const double kk = P.kscale * k;
        X = make_double2(kk * X.y, -kk * X.x);
      }
      acc = t == 0 ? X : cadd(acc, X);
    }
    const double sc = 0.5 * ((k == 0) ? J.s0 : J.s);
    double2 out = cscale(acc, sc);
    if (k == 0) out.y = 0.0;
    J.cout[(size_t)(row0 + c) * Kx + k] = out;
  }
}

inline size_t xfftm_smem(int L, int Kx, int nb) { return sizeof(double2) * (size_t)nb * (4 * L + Kx); }
constexpr int kXRowsMax = 4;

// Launch variant of the x transforms: rows per CTA nb (low byte) and threads per CTA nt (the
// bits above; 0 = 64).  nb = 1 with 64 threads is xfft_kernel, everything else xfftm_kernel.
// Threads per CTA that are a multiple of the butterflies of a pass keep every lane busy in
// it: for L = 192 (radix 4, 4, 4, 3: 48, 48, 48, 64 butterflies per row) that is 96 threads
// on two rows or 192 on four.
constexpr int xvar(int nb, int nt) { return nb | (nt << 8); }
constexpr int xvar_rows(int xv) { return xv & 0xff; }
constexpr int xvar_threads(int xv) { return (xv >> 8) ? (xv >> 8) : 64; }

// x-transform jobs over nrows rows in launch variant xv
inline cudaError_t launch_xfft(bool pdl, int xv, const XJobs& js, const XParams& xp, int nrows, cudaStream_t st) {
  const int nb = xvar_rows(xv) < 1 ? 1 : xvar_rows(xv), nt = xvar_threads(xv);
  if (nb == 1 && nt == 64)
    return launch_kernel(pdl, xfft_kernel, dim3(nrows, js.n), dim3(64), xfftm_smem(xp.L, xp.Kx, 1), st, js, xp);
  return launch_kernel(pdl, xfftm_kernel, dim3((nrows + nb - 1) / nb, js.n), dim3(nt), xfftm_smem(xp.L, xp.Kx, nb), st,
                       js, xp, nb, nrows);
}

// Launch variant for the x transforms of this problem: rows `forced` (1, 2 or 4, 64 threads)
// or, when 0, the fastest of the candidates below on the problem's own job set (timed with
// CUDA events, first run of each discarded).  Also raises the shared-memory limit of the
// kernels when needed.
inline int tune_xfft_rows(const XJobs& js, const XParams& xp, int nrows, cudaStream_t st, int forced,
                          cudaError_t* err) {
  *err = cudaSuccess;
  // row counts whose shared memory fits one CTA (raising the opt-in limit where needed)
  bool ok[kXRowsMax + 1] = {false, false, false, false, false};
  for (int nb : {1, 2, 4}) {
    const size_t sm = xfftm_smem(xp.L, xp.Kx, nb);
    if (sm <= 48 * 1024) {
      ok[nb] = true;
    } else if (sm <= 227 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(xfftm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e == cudaSuccess && nb == 1)
        e = cudaFuncSetAttribute(xfft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      ok[nb] = e == cudaSuccess;
      cudaGetLastError();
    }
  }
  if (forced == 1 || forced == 2 || forced == 4) return xvar(forced, 64);
  if (!ok[1]) return xvar(1, 64);  // rows too long for any variant: launches will report the error
  cudaEvent_t a = nullptr, b = nullptr;
  if ((*err = cudaEventCreate(&a)) != cudaSuccess) return xvar(1, 64);
  if ((*err = cudaEventCreate(&b)) != cudaSuccess) { cudaEventDestroy(a); return xvar(1, 64); }
  int best_xv = xvar(1, 64);
  float best = 1e30f;
  constexpr int cand[] = {xvar(1, 64), xvar(2, 64), xvar(4, 64), xvar(2, 96), xvar(4, 96), xvar(4, 128), xvar(4, 192)};
  // each candidate: one untimed launch, then the median of 7 timed ones (a lucky or unlucky single
  // launch does not decide the variant)
  for (int xv : cand) {
    if (!ok[xvar_rows(xv)]) continue;
    float t[7];
    int nt = 0;
    for (int rep = 0; rep < 8 && *err == cudaSuccess; ++rep) {
      cudaEventRecord(a, st);
      *err = launch_xfft(false, xv, js, xp, nrows, st);
      cudaEventRecord(b, st);
      if (*err == cudaSuccess) *err = cudaEventSynchronize(b);
      float ms = 0.f;
      if (*err == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
      if (rep > 0) t[nt++] = ms;
    }
    if (nt == 7) {
      std::sort(t, t + 7);
      if (t[3] < best) { best = t[3]; best_xv = xv; }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best_xv;
}

// Grid-field slots: 0 u, 1 ux, 2 uz, 3 w, 4 wx, 5 wz, 6 tx, 7 tz (the forward and tangent
// products are formed inside xfft_kernel from product specs; the reverse products have their
// own kernel).
// Reverse of the products F_u = -(u ux + w uz), F_w = -(u wx + w wz), F_t = -(u tx + w tz):
// from grid cotangents (gu, gw, gt) of (F_u, F_w, F_t) produce the
// cotangents of the 8 grid fields.
__global__ void prod_vjp_kernel(const double* __restrict__ G, const double* __restrict__ gF, double* __restrict__ Gb,
                                int npts) {
  pdl_trigger();
  pdl_wait();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npts; i += gridDim.x * blockDim.x) {
    const double u = G[0 * (size_t)npts + i], ux = G[1 * (size_t)npts + i], uz = G[2 * (size_t)npts + i];
    const double w = G[3 * (size_t)npts + i], wx = G[4 * (size_t)npts + i], wz = G[5 * (size_t)npts + i];
    const double tx = G[6 * (size_t)npts + i], tz = G[7 * (size_t)npts + i];
    const double gu = gF[0 * (size_t)npts + i], gw = gF[1 * (size_t)npts + i], gt = gF[2 * (size_t)npts + i];
    Gb[0 * (size_t)npts + i] = -(gu * ux + gw * wx + gt * tx);
    Gb[1 * (size_t)npts + i] = -gu * u;
    Gb[2 * (size_t)npts + i] = -gu * w;
    Gb[3 * (size_t)npts + i] = -(gu * uz + gw * wz + gt * tz);
    Gb[4 * (size_t)npts + i] = -gw * u;
    Gb[5 * (size_t)npts + i] = -gw * w;
    Gb[6 * (size_t)npts + i] = -gt * u;
    Gb[7 * (size_t)npts + i] = -gt * w;
  }
}

// Stage solve x = Phi v per pencil and parity class (or the adjoint v = Phi^H x), with the
// right-hand side formed on the fly as v = sum_t a_t in_t.  Phi = Dc Phi' Dr with real
// Phi' stored per pencil as two (3N/2)^2 parity blocks, once as [k][r] = Phi'[r][k] (read by
// the forward map) and once as [k][r] = Phi'[k][r] (read by the adjoint map), so that the
// threads of a warp, which own consecutive output rows r, read consecutive addresses.  Dr,
// Dc^H and the projection of the mean pencil onto real coefficients are applied on load and
// store.  CTA = (pencil, class, half of the rows); thread = (row, quarter of the columns).  The
// CTA's rows of the operator are staged in shared memory by cp.async before the kernel waits
// for its predecessor (programmatic dependent launch), so the staging overlaps that kernel.
struct SolveArgs {
  const double2* in[16];
  double a[16];
  int nin;
  double2* out;
  double2* vout;  // nullable: the combined operand sum_t a_t in_t is also stored here (forward only)
  int transpose;
  const double* phiF;  // [Kx][2][H][H] as [k][r] = Phi'[r][k]
  const double* phiA;  // [Kx][2][H][H] as [k][r] = Phi'[k][r]
  int Kx, N;
};

__host__ __device__ inline int solve_rows(int H) { return (H + 1) / 2; }

__global__ void __launch_bounds__(1024) solve_kernel(const __grid_constant__ SolveArgs S) {
  pdl_trigger();
  const int m = blockIdx.x, cls = blockIdx.y;
  const int N = S.N, Nh = N / 2, H = 3 * Nh, Kx = S.Kx;
  const int RH = solve_rows(H);
  const int r0 = blockIdx.z * RH;
  const int nr = min(RH, H - r0);
  extern __shared__ double2 sv[];  // v[H], red[4][RH], then this CTA's operator rows ph[H][RH]
  double2* v = sv;
  double2* red = sv + H;
  double* ph = reinterpret_cast<double*>(sv + H + 4 * RH);
  const double* blk = (S.transpose ? S.phiA : S.phiF) + ((size_t)m * 2 + cls) * H * H;
  const int tid = threadIdx.x, nt = blockDim.x;
  // the operator does not depend on the preceding kernels: stage it while they finish
  for (int idx = tid; idx < H * nr; idx += nt) {
    const int k = idx / nr, rl = idx - k * nr;
    cp_async8(ph + (size_t)k * RH + rl, blk + (size_t)k * H + r0 + rl);
  }
  cp_async_commit();
  pdl_wait();
  // class index c -> (field f, mode n)
  for (int c = tid; c < H; c += nt) {
    const int f = c / Nh, h = c % Nh;
    const int n = 2 * h + ((f == 0) ? cls : 1 - cls);
    const size_t off = ((size_t)f * Kx + m) * N + n;
    double2 x = make_double2(0.0, 0.0);
    for (int t = 0; t < S.nin; ++t) {
      const double2 y = S.in[t][off];
      x.x = fma(S.a[t], y.x, x.x);
      x.y = fma(S.a[t], y.y, x.y);
    }
    if (S.vout && blockIdx.z == 0) S.vout[off] = x;  // one row block of each (pencil, class) stores it
    if (S.transpose && m == 0) x.y = 0.0;          // projection (self-adjoint)
    if (f == 0) x = make_double2(x.y, -x.x);        // times -i (Dr, or Dc^H)
    v[c] = x;
  }
  cp_async_wait_all();
  __syncthreads();
  const int rl = tid % RH, q = tid / RH;
  const int r = r0 + rl;
  const int kq = (H + 3) / 4;
  const int k0 = q * kq, k1 = min(H, k0 + kq);
  double2 acc0 = make_double2(0.0, 0.0), acc1 = make_double2(0.0, 0.0);
  if (r < H && q < 4) {
    int k = k0;
    for (; k + 1 < k1; k += 2) {
      const double p0 = ph[(size_t)k * RH + rl], p1 = ph[(size_t)(k + 1) * RH + rl];
      const double2 x0 = v[k], x1 = v[k + 1];
      acc0.x = fma(p0, x0.x, acc0.x); acc0.y = fma(p0, x0.y, acc0.y);
      acc1.x = fma(p1, x1.x, acc1.x); acc1.y = fma(p1, x1.y, acc1.y);
    }
    if (k < k1) {
      const double p0 = ph[(size_t)k * RH + rl];
      const double2 x0 = v[k];
      acc0.x = fma(p0, x0.x, acc0.x); acc0.y = fma(p0, x0.y, acc0.y);
    }
  }
  if (q < 4) red[q * RH + rl] = cadd(acc0, acc1);
  __syncthreads();
  if (tid < RH && r0 + tid < H) {
    double2 acc = red[tid];
    for (int qq = 1; qq < 4; ++qq) acc = cadd(acc, red[qq * RH + tid]);
    const int c = r0 + tid;
    const int f = c / Nh, h = c % Nh;
    const int n = 2 * h + ((f == 0) ? cls : 1 - cls);
    if (f == 0) acc = make_double2(-acc.y, acc.x);  // times i (Dc, or Dr^H)
    if (!S.transpose && m == 0) acc.y = 0.0;        // projection onto real mean pencil
    S.out[((size_t)f * Kx + m) * N + n] = acc;
  }
}

// Fused column stage of the RK222 forward step for one x-mode pencil, as a cluster of two
// CTAs (one per z-parity class, cluster rank = class):
//   1. fold: f = Gz Y for the three grid-product rows Y_q (mixed [Mz][Kx]) restricted to the
//      modes of this class (the reflection-folded Chebyshev reduction of zmm_kernel);
//   2. solve: x = Phi (sum_t a_t in_t + af f) for this class (solve_kernel's arithmetic), with
//      the class block of Phi' brought into shared memory by one bulk copy (cp.async.bulk,
//      completing on an mbarrier) issued at entry, so it lands during the fold;
//   3. when zout is set: the two CTAs exchange their halves of x through distributed shared
//      memory and each expands three of the six grid fields (u, dz u, w, dz w, theta,
//      dz theta; class 0 the values, class 1 the z-derivatives) into zout[6][Mz][Kx].
// f and x are also written in the state layout [3][Kx][N].  Replaces zmm fold + solve +
// zmm expand (three launches) by one.  The kernel is FP64-throughput bound (one thread per
// output of each phase keeps the dependency chains long but the FP64 pipe busy; spreading the dot
// products over all threads with a reduction measured slower, its adds cost FP64 issue slots).
// A bulk copy that does not complete within the bounded wait sets *err (the launch's results are
// then invalid; the host reports it).
struct ColStepArgs {
  const double2* yin[3];  // grid products after the x-forward FFT, mixed layout
  const double* gzF;      // N x (Mz/2) fold matrix
  double2* f_out;
  const double2* in[4];
  double a[4];
  int nin;
  double af;
  const double* phiF;     // [Kx][2][H][H] as [k][r]
  double2* x_out;
  const double* czE;      // (Mz/2) x N
  const double* cdzE;     // (Mz/2) x N (z-derivative parity)
  double2* zout;          // nullable
  size_t nmix;
  int Kx, N, Mz;
  int* err;
  int bulk;               // 1: operator block by one bulk copy; 0: per-thread cp.async
};

constexpr unsigned kCsSpin = 1u << 20;  // bounded wait for the operator block's bulk copy

// Bounded wait of every thread for the operator block; a second bounded wait after a timeout
// (the copy targets this CTA's shared memory, which must not be left while it may still land).
__device__ __forceinline__ void colstep_wait_block(unsigned long long* bar, int* err, int bulk) {
  if (!bulk) {
    cp_async_wait_all();
    return;
  }
  if (!mbar_wait_bounded(bar, 0, kCsSpin, err)) mbar_wait_bounded(bar, 0, kCsSpin, nullptr);
}

// The class block (H x H doubles) into ph: one bulk copy counted on bar (thread 0), or, when
// bulk == 0, 16-byte cp.async copies spread over the threads (completed by colstep_wait_block).
__device__ __forceinline__ void colstep_issue_block(double* ph, const double* blk, int H, unsigned long long* bar,
                                                    int bulk) {
  if (bulk) {
    if (threadIdx.x == 0) {
      const unsigned bytes = (unsigned)(sizeof(double) * (size_t)H * H);
      mbar_init(bar, 1);
      mbar_arrive_expect_tx(bar, bytes);
      bulk_g2s(ph, blk, bytes, bar);
    }
  } else {
    for (int idx = threadIdx.x; idx < H * H / 2; idx += blockDim.x)
      cp_async16(reinterpret_cast<double2*>(ph) + idx, reinterpret_cast<const double2*>(blk) + idx);
    cp_async_commit();
  }
}

__host__ __device__ inline size_t colstep_smem(int N, int Mz) {
  const int H = 3 * N / 2;
  return sizeof(double) * (size_t)H * H + sizeof(double2) * (size_t)(3 * (Mz / 2) + 3 * N + H + H);
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(256) rb_colstep_kernel(const __grid_constant__ ColStepArgs S) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int cls = (int)cluster.block_rank();
  const int m = blockIdx.x >> 1;
  const int N = S.N, Nh = N / 2, H = 3 * Nh, Kx = S.Kx, Mz = S.Mz, Mh = Mz / 2;
  const int tid = threadIdx.x, nt = blockDim.x;
  extern __shared__ double2 cs[];
  __shared__ unsigned long long bar;
  double* ph = reinterpret_cast<double*>(cs);          // [H][H] as [k][r]
  double2* sd = cs + (size_t)H * H / 2;                // [3][Mh] folded samples (s or d)
  double2* fs = sd + 3 * Mh;                           // [3][N] f (this class's modes)
  double2* v = fs + 3 * N;                             // [H] right-hand side (class order)
  double2* xc = v + H;                                 // [H] solution (class order)
  colstep_issue_block(ph, S.phiF + ((size_t)m * 2 + cls) * H * H, H, &bar, S.bulk);
  pdl_trigger();
  pdl_wait();
  // class-local mode of field q: parity (q == 0 ? cls : 1 - cls); fold with s (even) or d (odd)
  for (int idx = tid; idx < 3 * Mh; idx += nt) {
    const int q = idx / Mh, j = idx - q * Mh;
    const int par = (q == 0) ? cls : 1 - cls;
    const double2 a = S.yin[q][(size_t)j * Kx + m], b = S.yin[q][(size_t)(Mz - 1 - j) * Kx + m];
    sd[idx] = par == 0 ? make_double2(a.x + b.x, a.y + b.y) : make_double2(a.x - b.x, a.y - b.y);
  }
  __syncthreads();
  for (int idx = tid; idx < 3 * Nh; idx += nt) {
    const int q = idx / Nh, h = idx - q * Nh;
    const int n = 2 * h + ((q == 0) ? cls : 1 - cls);
    const double* g = S.gzF + (size_t)n * Mh;
    const double2* w = sd + q * Mh;
    double2 a0 = make_double2(0.0, 0.0), a1 = make_double2(0.0, 0.0);
    int j = 0;
    for (; j + 1 < Mh; j += 2) {
      const double g0 = __ldg(g + j), g1 = __ldg(g + j + 1);
      a0.x = fma(g0, w[j].x, a0.x); a0.y = fma(g0, w[j].y, a0.y);
      a1.x = fma(g1, w[j + 1].x, a1.x); a1.y = fma(g1, w[j + 1].y, a1.y);
    }
    if (j < Mh) {
      const double g0 = __ldg(g + j);
      a0.x = fma(g0, w[j].x, a0.x); a0.y = fma(g0, w[j].y, a0.y);
    }
    const double2 f = cadd(a0, a1);
    fs[q * N + n] = f;
    S.f_out[((size_t)q * Kx + m) * N + n] = f;
  }
  __syncthreads();
  for (int c = tid; c < H; c += nt) {
    const int q = c / Nh, h = c % Nh;
    const int n = 2 * h + ((q == 0) ? cls : 1 - cls);
    const size_t off = ((size_t)q * Kx + m) * N + n;
    const double2 f = fs[q * N + n];
    double2 x = make_double2(S.af * f.x, S.af * f.y);
    for (int t = 0; t < S.nin; ++t) {
      const double2 y = S.in[t][off];
      x.x = fma(S.a[t], y.x, x.x);
      x.y = fma(S.a[t], y.y, x.y);
    }
    if (q == 0) x = make_double2(x.y, -x.x);  // times -i (Dr)
    v[c] = x;
  }
  colstep_wait_block(&bar, S.err, S.bulk);
  __syncthreads();
  for (int r = tid; r < H; r += nt) {
    double2 a0 = make_double2(0.0, 0.0), a1 = make_double2(0.0, 0.0);
    int k = 0;
    for (; k + 1 < H; k += 2) {
      const double p0 = ph[(size_t)k * H + r], p1 = ph[(size_t)(k + 1) * H + r];
      const double2 x0 = v[k], x1 = v[k + 1];
      a0.x = fma(p0, x0.x, a0.x); a0.y = fma(p0, x0.y, a0.y);
      a1.x = fma(p1, x1.x, a1.x); a1.y = fma(p1, x1.y, a1.y);
    }
    if (k < H) {
      const double p0 = ph[(size_t)k * H + r];
      a0.x = fma(p0, v[k].x, a0.x); a0.y = fma(p0, v[k].y, a0.y);
    }
    double2 acc = cadd(a0, a1);
    const int q = r / Nh, h = r % Nh;
    const int n = 2 * h + ((q == 0) ? cls : 1 - cls);
    if (q == 0) acc = make_double2(-acc.y, acc.x);  // times i (Dc)
    if (m == 0) acc.y = 0.0;                        // projection onto the real mean pencil
    xc[r] = acc;
    S.x_out[((size_t)q * Kx + m) * N + n] = acc;
  }
  if (!S.zout) return;
  cluster.sync();  // both halves of x are in shared memory
  const double2* xo = cluster.map_shared_rank(xc, 1 - cls);
  // expand: field q, value (cls 0) or z-derivative (cls 1); even/odd mode sums from the class
  // that holds them (modes of parity cls' are in CTA cls' = (q == 0 ? par : 1 - par))
  const double* Cm = cls == 0 ? S.czE : S.cdzE;
  for (int idx = tid; idx < 3 * Mh; idx += nt) {
    const int q = idx / Mh, j = idx - q * Mh;
    const double* crow = Cm + (size_t)j * N;
    // modes 2h (even) live in CTA (q == 0 ? 0 : 1), modes 2h + 1 (odd) in the other one
    const int even_cta = (q == 0) ? 0 : 1;
    const double2* xe = (even_cta == cls ? xc : xo) + q * Nh;
    const double2* xd = (even_cta == cls ? xo : xc) + q * Nh;
    double2 E = make_double2(0.0, 0.0), O = make_double2(0.0, 0.0);
    for (int h = 0; h < Nh; ++h) {
      const double ce = __ldg(crow + 2 * h), co = __ldg(crow + 2 * h + 1);
      const double2 e = xe[h], o = xd[h];
      E.x = fma(ce, e.x, E.x); E.y = fma(ce, e.y, E.y);
      O.x = fma(co, o.x, O.x); O.y = fma(co, o.y, O.y);
    }
    const double se = cls == 0 ? 1.0 : -1.0;  // reflection parity of T_n (values) or dT_n/dz
    double2* out = S.zout + (size_t)(2 * q + cls) * S.nmix;
    out[(size_t)j * Kx + m] = make_double2(E.x + O.x, E.y + O.y);
    out[(size_t)(Mz - 1 - j) * Kx + m] = make_double2(se * (E.x - O.x), se * (E.y - O.y));
  }
  cluster.sync();  // the partner's shared memory stays alive until both expansions are done
}

// Fused column stage of the RK222 adjoint step (the transpose of rb_colstep_kernel's chain)
// for one x-mode pencil, as a cluster of two CTAs (one per z-parity class):
//   1. fold: xb = Cz^T a_q + (Cz Dz)^T b_q + sum_a beta_a add_a for the six mixed rows
//      (a_u, b_u, a_w, b_w, a_t, b_t) restricted to this class's modes;
//   2. transposed solve: vb = Phi^H xb for this class (solve_kernel's transpose arithmetic),
//      the class block of Phi' brought into shared memory by one bulk copy (completing on an
//      mbarrier) issued at entry;
//   3. the two CTAs exchange their halves of vb through distributed shared memory and each
//      expands, for half of the Gauss rows, the three columns Gz^T (al0 c0 + al1 vb) into
//      zout[3][Mz][Kx] (the first transform of the next vector-Jacobian product).
// vb is also written in the state layout.  Replaces zmm fold + solve + zmm expand.
struct ColStepTArgs {
  const double2* yin[6];
  const double* czTF;    // N x (Mz/2)
  const double* cdzTF;   // N x (Mz/2), z-derivative parity
  const double2* add[2];
  double beta[2];
  int nadd;
  const double* phiA;    // [Kx][2][H][H] as [k][r] = Phi'[k][r]
  double2* v_out;
  const double2* c0;
  double al0, al1;
  const double* gzTE;    // (Mz/2) x N
  double2* zout;
  size_t nmix;
  int Kx, N, Mz;
  int* err;
  int bulk;
};

__host__ __device__ inline size_t colstepT_smem(int N, int Mz) {
  const int H = 3 * N / 2;
  return sizeof(double) * (size_t)H * H + sizeof(double2) * (size_t)(6 * (Mz / 2) + H + H + 3 * N);
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(256) rb_colstepT_kernel(const __grid_constant__ ColStepTArgs S) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int cls = (int)cluster.block_rank();
  const int m = blockIdx.x >> 1;
  const int N = S.N, Nh = N / 2, H = 3 * Nh, Kx = S.Kx, Mz = S.Mz, Mh = Mz / 2;
  const int tid = threadIdx.x, nt = blockDim.x;
  extern __shared__ double2 cs[];
  __shared__ unsigned long long bar;
  double* ph = reinterpret_cast<double*>(cs);   // [H][H] as [k][r]
  double2* sd = cs + (size_t)H * H / 2;         // [6][Mh] folded samples
  double2* xv = sd + 6 * Mh;                    // [H] right-hand side (class order)
  double2* vc = xv + H;                         // [H] solution (class order)
  colstep_issue_block(ph, S.phiA + ((size_t)m * 2 + cls) * H * H, H, &bar, S.bulk);
  pdl_trigger();
  pdl_wait();
  // row e = 2q + term: term 0 (values) folds with s for even modes, term 1 (z-derivative
  // parity) with s for odd modes; this class's modes of field q have parity (q == 0 ? cls : 1 - cls)
  for (int idx = tid; idx < 6 * Mh; idx += nt) {
    const int e = idx / Mh, j = idx - e * Mh;
    const int q = e >> 1, term = e & 1;
    const int par = (q == 0) ? cls : 1 - cls;
    const bool use_s = (par == 0) != (term == 1);
    const double2 a = S.yin[e][(size_t)j * Kx + m], b = S.yin[e][(size_t)(Mz - 1 - j) * Kx + m];
    sd[idx] = use_s ? make_double2(a.x + b.x, a.y + b.y) : make_double2(a.x - b.x, a.y - b.y);
  }
  __syncthreads();
  for (int c = tid; c < H; c += nt) {
    const int q = c / Nh, h = c % Nh;
    const int n = 2 * h + ((q == 0) ? cls : 1 - cls);
    const double* g0 = S.czTF + (size_t)n * Mh;
    const double* g1 = S.cdzTF + (size_t)n * Mh;
    const double2* w0 = sd + (2 * q) * Mh;
    const double2* w1 = sd + (2 * q + 1) * Mh;
    double2 a0 = make_double2(0.0, 0.0), a1 = make_double2(0.0, 0.0);
    for (int j = 0; j < Mh; ++j) {
      const double c0 = __ldg(g0 + j), c1 = __ldg(g1 + j);
      a0.x = fma(c0, w0[j].x, a0.x); a0.y = fma(c0, w0[j].y, a0.y);
      a1.x = fma(c1, w1[j].x, a1.x); a1.y = fma(c1, w1[j].y, a1.y);
    }
    double2 x = cadd(a0, a1);
    const size_t off = ((size_t)q * Kx + m) * N + n;
    for (int a = 0; a < S.nadd; ++a) {
      const double2 y = S.add[a][off];
      x.x = fma(S.beta[a], y.x, x.x);
      x.y = fma(S.beta[a], y.y, x.y);
    }
    if (m == 0) x.y = 0.0;                     // projection (self-adjoint)
    if (q == 0) x = make_double2(x.y, -x.x);  // times -i (Dc^H)
    xv[c] = x;
  }
  colstep_wait_block(&bar, S.err, S.bulk);
  __syncthreads();
  for (int r = tid; r < H; r += nt) {
    double2 a0 = make_double2(0.0, 0.0), a1 = make_double2(0.0, 0.0);
    int k = 0;
    for (; k + 1 < H; k += 2) {
      const double p0 = ph[(size_t)k * H + r], p1 = ph[(size_t)(k + 1) * H + r];
      const double2 x0 = xv[k], x1 = xv[k + 1];
      a0.x = fma(p0, x0.x, a0.x); a0.y = fma(p0, x0.y, a0.y);
      a1.x = fma(p1, x1.x, a1.x); a1.y = fma(p1, x1.y, a1.y);
    }
    if (k < H) {
      const double p0 = ph[(size_t)k * H + r];
      a0.x = fma(p0, xv[k].x, a0.x); a0.y = fma(p0, xv[k].y, a0.y);
    }
    double2 acc = cadd(a0, a1);
    const int q = r / Nh, h = r % Nh;
    const int n = 2 * h + ((q == 0) ? cls : 1 - cls);
    if (q == 0) acc = make_double2(-acc.y, acc.x);  // times i (Dr^H)
    vc[r] = acc;
    S.v_out[((size_t)q * Kx + m) * N + n] = acc;
  }
  cluster.sync();
  const double2* vo = cluster.map_shared_rank(vc, 1 - cls);
  // the expanded vector al0 c0 + al1 v of each field, even (cx[q][0][h]) and odd (cx[q][1][h])
  // modes, formed once here instead of once per output row
  double2* cx = vc + H;  // [3][2][Nh]
  for (int idx = tid; idx < 3 * N; idx += nt) {
    const int q = idx / N, par = (idx / Nh) & 1, h = idx % Nh;
    const int even_cta = (q == 0) ? 0 : 1;
    const double2* v = ((even_cta == cls) == (par == 0) ? vc : vo) + q * Nh;
    const double2 c = S.c0[((size_t)q * Kx + m) * N + 2 * h + par];
    cx[idx] = make_double2(fma(S.al0, c.x, S.al1 * v[h].x), fma(S.al0, c.y, S.al1 * v[h].y));
  }
  __syncthreads();
  const int jh = (Mh + 1) / 2;
  const int j0 = cls == 0 ? 0 : jh, j1 = cls == 0 ? jh : Mh;
  for (int idx = tid; idx < 3 * (j1 - j0); idx += nt) {
    const int q = idx / (j1 - j0), j = j0 + idx % (j1 - j0);
    const double* grow = S.gzTE + (size_t)j * N;
    const double2* xe = cx + (size_t)q * N;
    const double2* xo = xe + Nh;
    double2 E = make_double2(0.0, 0.0), O = make_double2(0.0, 0.0);
    for (int h = 0; h < Nh; ++h) {
      const double ge = __ldg(grow + 2 * h), go = __ldg(grow + 2 * h + 1);
      E.x = fma(ge, xe[h].x, E.x); E.y = fma(ge, xe[h].y, E.y);
      O.x = fma(go, xo[h].x, O.x); O.y = fma(go, xo[h].y, O.y);
    }
    double2* out = S.zout + (size_t)q * S.nmix;
    out[(size_t)j * Kx + m] = make_double2(E.x + O.x, E.y + O.y);
    out[(size_t)(Mz - 1 - j) * Kx + m] = make_double2(E.x - O.x, E.y - O.y);
  }
  cluster.sync();
}

// Kinetic energy J = (Lx/2) sum_{u,w} sum_m w_m c_m^H G c_m and its gradient
// seed = Lx w_m G c_m (w_0 = 1, w_m = 2; real part only on the mean pencil).
__global__ void energy_kernel(const double2* __restrict__ x, const double* __restrict__ G, double Lx, int Kx, int N,
                              double* __restrict__ partial, double2* __restrict__ seed) {
  const int m = blockIdx.x;
  const double wm = (m == 0) ? 1.0 : 2.0;
  double acc = 0.0;
  for (int idx = threadIdx.x; idx < 3 * N; idx += blockDim.x) {
    const int f = idx / N, i = idx % N;
    const size_t base = ((size_t)f * Kx + m) * N;
    double2 g = make_double2(0.0, 0.0);
    if (f < 2) {
      for (int k = 0; k < N; ++k) {
        double2 c = x[base + k];
        if (m == 0) c.y = 0.0;
        const double gv = __ldg(&G[i * N + k]);
        g.x = fma(gv, c.x, g.x);
        g.y = fma(gv, c.y, g.y);
      }
      double2 ci = x[base + i];
      if (m == 0) ci.y = 0.0;
      acc += ci.x * g.x + ci.y * g.y;
    }
    seed[base + i] = make_double2(Lx * wm * g.x, Lx * wm * g.y);
  }
  __shared__ double red[128];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[m] = 0.5 * Lx * wm * red[0];
}

__global__ void sum_kernel(const double* __restrict__ partial, int n, double* __restrict__ out) {
  __shared__ double red[128];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += partial[i];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// y = sum_t a_t x_t over n complex entries (state combinations).
// Linear combinations of state vectors in one launch.  combine: out = a_0 in_0 + a_1 in_1 + ...
// (in_0 may be out; the terms are added by multiply-adds in term order, the same sums as a chain
// of axpy_kernel launches); scatter: out_k += c_k src for several distinct outputs (none equal to
// src).
constexpr int kCombMax = 16;
struct CombArgs {
  const double2* in[kCombMax];
  double a[kCombMax];
  int n;
  double2* out;
  size_t count;
};
__global__ void combine_kernel(const __grid_constant__ CombArgs A) {
  pdl_trigger();
  pdl_wait();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < A.count; i += (size_t)gridDim.x * blockDim.x) {
    double2 v = A.in[0][i];
    double2 r = make_double2(A.a[0] * v.x, A.a[0] * v.y);
    for (int t = 1; t < A.n; ++t) {
      v = A.in[t][i];
      r.x = fma(A.a[t], v.x, r.x);
      r.y = fma(A.a[t], v.y, r.y);
    }
    A.out[i] = r;
  }
}
struct ScatArgs {
  double2* out[kCombMax];
  double c[kCombMax];
  int n;
  const double2* src;
  size_t count;
};
__global__ void scatter_kernel(const __grid_constant__ ScatArgs A) {
  pdl_trigger();
  pdl_wait();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < A.count; i += (size_t)gridDim.x * blockDim.x) {
    const double2 s = A.src[i];
    for (int k = 0; k < A.n; ++k) {
      double2 y = A.out[k][i];
      y.x = fma(A.c[k], s.x, y.x);
      y.y = fma(A.c[k], s.y, y.y);
      A.out[k][i] = y;
    }
  }
}

__global__ void axpy_kernel(double2* __restrict__ y, const double2* __restrict__ x0, double a0,
                            const double2* __restrict__ x1, double a1, const double2* __restrict__ x2, double a2,
                            size_t n) {
  pdl_trigger();
  pdl_wait();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double2 v = x0[i];
    double2 r = make_double2(a0 * v.x, a0 * v.y);
    if (x1) { v = x1[i]; r.x = fma(a1, v.x, r.x); r.y = fma(a1, v.y, r.y); }
    if (x2) { v = x2[i]; r.x = fma(a2, v.x, r.x); r.y = fma(a2, v.y, r.y); }
    y[i] = r;
  }
}

}  // namespace
}  // namespace rbk
}  // namespace spadj
