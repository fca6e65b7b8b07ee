// Batched 2D Kolmogorov flow (vorticity form, Fourier x Fourier, SBDF1 -> SBDF2) with 4D-Var
// gradients: every member of a mixed-resolution batch advances in ONE persistent launch.
//
// Per member and timestep the work splits into tiles of two kinds:
//   CA (column tile, a few x-modes): finish step s for these x-modes -- y-FFT of the grid
//      product, IMEX combination of eq. imex with the diagonal implicit solve, projection onto
//      admissible coefficients -- then start step s+1 for the same x-modes: the spectral fields
//      u, v, w_x, w_y (u = i ky w/|k|^2, v = -i kx w/|k|^2) and their inverse y-FFTs.
//   B  (row tile, a few grid rows in y): inverse x-FFTs of the four fields, the product
//      u w_x + v w_y on the dealiased grid, forward x-FFT.
// Within a member, CA of step s+1 needs every B tile of step s and B of step s needs every CA
// tile of step s; nothing else is shared, so members of different sizes interleave freely.
// The adjoint (eq. IMEX_adjoint) has the same two-kind structure: C'A' tiles finish the VJP
// of F, add the injected 4D-Var cotangents, solve for Y_n and start the next VJP (T^dagger of
// the cotangent, fields of X_{n-1} from the stored trajectory); B' tiles do the grid products
// of the VJP and the adjoint x-FFTs.
//
// Scheduler: work items (stage, phase, member, tile) are handed out in order from a global
// counter to a grid of resident CTAs (occupancy-sized, so every CTA holding an item runs); an
// item waits, with a bounded spin, for the per-member completion counter of the phase it
// depends on.  A wait that exceeds its limit sets an error flag, every CTA stops, and the host
// returns SPADJ_ERR_TIMEOUT.  Data produced inside the launch is read with ld.global.cg.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "closure.cuh"
#include "fft.cuh"
#include "problem.h"

namespace spadj {
namespace {

constexpr int kKolThreads = 128;
constexpr int kMaxRes = 4;
constexpr unsigned kSpinLimit = 1u << 26;  // x ~150 ns per probe: several seconds

struct KMember {
  int N, Kx, M, L, res;
  long long off_state;  // complex offset of the member in a state array
  long long off_mix;    // complex offset of the member in a mixed [y][kx] array
  long long off_grid;   // offset of the member in a real [y][x] grid array
  int nCA, nB;          // tiles per stage
  int caStart, bStart;  // first item of the member inside a stage's CA / B block
};

struct KRes {
  FFTPlan px, py;
  const double2* WMx;  // exp(-2 pi i m / M), m < M  (x real FFT through L = M/2)
  const double2* W2M;  // exp(-2 pi i m / 2M), m < 2M (y complex FFT of length M)
};

struct KolArgs {
  int nmem;
  const KMember* mem;
  KRes res[kMaxRes];
  double Re, dt;
  double invRe;      // 1 / Re
  double kc[2][5];   // SBDF1 (row 0) and SBDF2 (row 1): a0, a1, a2 (divided by dt), c1, c2
  int CW, RW;
  int nCAtot, nBtot;
  int adjoint;      // 0 forward, 1 adjoint
  int fonly;        // forward: stage-0 F evaluation only (writes F(x0) to out)
  int nstage;       // number of stages in this launch
  // persistent launch over stages stage0 .. stage0 + nrun - 1 of the sweep only (nrun = 0: all); the
  // completion counters count from the sweep's first stage, so a later launch waits on the same targets
  int stage0, nrun;
  int S;            // n_steps of the sweep (adjoint: the horizon N, which fixes the weights and the seed)
  // Segments (checkpointed sweeps).  Forward: stage s is step n0 + s (x0 = X_{n0}, with X_{n0-1} and
  // F(X_{n0-1}) preset in the rings when n0 >= 1), traj (nullable) holds the launch's states relative
  // to n0.  Adjoint: stage k processes index n0 - k; prologue = 1: stage 0 only forms the transforms
  // of W_{n0-1} from Y_{n0}, Y_{n0+1} in the Y ring (the second half of index n0, whose first half ran
  // in the previous launch); lo: lowest index of the launch (its second half is skipped when lo > 0),
  // traj holds X_lo .. (relative to lo).
  int n0;
  int prologue;
  int lo;
  int forcing, nonlinear;
  const double2* x0;
  double2* Xr[2];
  double2* Fr[2];
  double2* Yr[2];
  double2* mixA[6];
  double2* mixB[5];
  int closure;            // learned closure active: omega itself is carried as a fifth field
  double* gridW;          // closure input grid (vorticity), [member][y][x]
  double* gridG;          // adjoint: T^dagger of the cotangent on the grid
  double2* traj;
  double2* out;
  const int* seed_at;
  const double2* seeds;
  long long state_size;
  int* queue;
  int* caDone;
  int* bDone;
  int* err;
  int smem_entries;       // dynamic shared memory of a CTA, in double2
  unsigned spin_limit;    // bounded-wait iterations
  int drop_signal_member; // test knob: completion of this member is never signalled (-1: off)
};

__device__ __forceinline__ double2 ldcg2(const double2* p) { return __ldcg(p); }

struct Coef {
  double a0, a1, a2, c1, c2;
};
// SBDF1 at n = 1, SBDF2 after; the weights come divided by dt from the host (no division here)
__device__ __forceinline__ Coef kcoef(int n, const double (&kc)[2][5]) {
  const double* w = kc[n <= 1 ? 0 : 1];
  return Coef{w[0], w[1], w[2], w[3], w[4]};
}

// ky of coefficient row q, and its index in the length-M y-FFT (-1 for the unstored Nyquist)
__device__ __forceinline__ int kyof(int q, int N) { return q < N / 2 ? q : q - N; }
__device__ __forceinline__ int yidx(int q, int N, int M) { return q < N / 2 ? q : (q == N / 2 ? -1 : M - N + q); }

// multiplier of field f (0 u, 1 v, 2 w_x, 3 w_y) applied to w(kx, ky)
__device__ __forceinline__ double2 fmult(int f, double kx, double ky, double2 w) {
  const double k2 = kx * kx + ky * ky;
  const double ik2 = k2 > 0.0 ? 1.0 / k2 : 0.0;
  double s;
  switch (f) {
    case 0: s = ky * ik2; break;    // i ky / |k|^2
    case 1: s = -kx * ik2; break;   // -i kx / |k|^2
    case 2: s = kx; break;          // i kx
    default: s = ky; break;         // i ky
  }
  return make_double2(-s * w.y, s * w.x);  // i s w
}

// project a column held in smem: Nyquist row to zero; kx = 0 column Hermitian
__device__ void project_col(double2* x, int N, int kx) {
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    if (q == N / 2) { x[q] = make_double2(0.0, 0.0); continue; }
    if (kx != 0) continue;
    const int p = (N - q) % N;
    if (q == 0) { x[0].y = 0.0; continue; }
    if (q < p) {
      const double2 a = x[q], b = x[p];
      const double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
      x[q] = h;
      x[p] = make_double2(h.x, -h.y);
    }
  }
  __syncthreads();
}

// y-FFT of a padded column: fill a (length M) from fill(j), transform with SIGN, return result
template <int SIGN>
__device__ double2* col_fft(double2* a, double2* b, const KRes& R) {
  __syncthreads();
  return cfft_smem_t<SIGN>(a, b, R.py, R.W2M);
}

struct KSmem {
  double2* buf;  // base of dynamic smem
};

// ---- forward CA tile --------------------------------------------------------------------------
__device__ void ca_forward(const KolArgs& A, const KMember& m, int tile, int s) {
  extern __shared__ double2 ks[];
  const int N = m.N, Kx = m.Kx, M = m.M;
  const int n = A.n0 + s;           // absolute step of this stage
  const int last = A.nstage - 1;    // the launch's last stage
  const KRes& R = A.res[m.res];
  double2* ca = ks;          // M
  double2* cb = ca + M;      // M
  double2* xc = cb + M;      // N
  const int kx0 = tile * A.CW, kx1 = min(Kx, kx0 + A.CW);
  const long long S = A.state_size;
  for (int kx = kx0; kx < kx1; ++kx) {
    const long long col = m.off_state + (long long)kx * N;
    if (s == 0) {
      for (int q = threadIdx.x; q < N; q += blockDim.x) xc[q] = A.x0[col + q];
      __syncthreads();
    } else {
      double2* r = nullptr;
      if (A.nonlinear || A.closure) {
        for (int j = threadIdx.x; j < M; j += blockDim.x) ca[j] = ldcg2(&A.mixB[0][m.off_mix + (long long)j * Kx + kx]);
        r = col_fft<-1>(ca, cb, R);
      }
      const Coef c = kcoef(n, A.kc);
      const double invM = 1.0 / M;
      for (int q = threadIdx.x; q < N; q += blockDim.x) {
        const int idx = yidx(q, N, M);
        const double ky = kyof(q, N);
        double2 F = make_double2(0.0, 0.0);
        if (idx >= 0 && (A.nonlinear || A.closure)) F = make_double2(-r[idx].x * invM, -r[idx].y * invM);
        if (A.forcing && kx == 0 && (q == 4 || q == N - 4)) F.x -= 2.0;
        if (A.fonly) {
          A.out[col + q] = F;
          continue;
        }
        const double2 X1 = ldcg2(&A.Xr[(n - 1) & 1][col + q]);
        double2 num = make_double2(c.c1 * F.x - c.a1 * X1.x, c.c1 * F.y - c.a1 * X1.y);
        if (n >= 2) {
          const double2 X2 = ldcg2(&A.Xr[n & 1][col + q]);
          const double2 F2 = ldcg2(&A.Fr[n & 1][col + q]);
          num.x += c.c2 * F2.x - c.a2 * X2.x;
          num.y += c.c2 * F2.y - c.a2 * X2.y;
        }
        A.Fr[(n - 1) & 1][col + q] = F;
        const double inv = 1.0 / (c.a0 + ((double)kx * kx + ky * ky) * A.invRe);
        xc[q] = make_double2(num.x * inv, num.y * inv);
      }
      __syncthreads();
      if (A.fonly) continue;
      project_col(xc, N, kx);
    }
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
      A.Xr[n & 1][col + q] = xc[q];
      if (A.traj) A.traj[(long long)s * S + col + q] = xc[q];
      if (s == last) A.out[col + q] = xc[q];
    }
    if (s < last && (A.nonlinear || A.closure)) {
      // the fields' inverse y transforms two at a time, sharing their passes: set p at
      // ks + 2 p M (scratch + M); the column is read back from the state just written, its
      // shared slot being reused
      const int nf = A.closure ? 5 : 4;
      const double2* xs = A.Xr[n & 1] + col;
      for (int f0 = 0; f0 < nf; f0 += 2) {
        const int np = min(2, nf - f0);
        __syncthreads();
        for (int i = threadIdx.x; i < np * M; i += blockDim.x) {
          const int pq = i / M;
          ks[pq * 2 * M + (i - pq * M)] = make_double2(0.0, 0.0);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < np * N; i += blockDim.x) {
          const int pq = i / N, q = i - pq * N, f = f0 + pq;
          const int idx = yidx(q, N, M);
          if (idx < 0) continue;
          const double2 x = ldcg2(&xs[q]);
          ks[pq * 2 * M + idx] = f < 4 ? fmult(f, (double)kx, (double)kyof(q, N), x) : x;
        }
        __syncthreads();
        cfft_smem_sets<1>(ks, ks + M, 2 * M, np, R.py, 1);
        const double2* r = (R.py.nrad & 1) ? ks + M : ks;
        for (int i = threadIdx.x; i < np * M; i += blockDim.x) {
          const int pq = i / M, j = i - pq * M;
          A.mixA[f0 + pq][m.off_mix + (long long)j * Kx + kx] = r[pq * 2 * M + j];
        }
      }
    }
    __syncthreads();
  }
}

// inverse x transform of one mixed row into a packed real row (L complex) kept in dst
__device__ void row_c2r(const double2* src, double2* dst, double2* sa, double2* sb, double2* st, const KMember& m,
                        const KRes& R, double w0, double w) {
  const int Kx = m.Kx, L = m.L;
  for (int k = threadIdx.x; k < Kx; k += blockDim.x) st[k] = ldcg2(&src[k]);
  __syncthreads();
  c2r_pre(sa, [&](int k) { return st[k]; }, Kx, L, R.WMx, w0, w);
  __syncthreads();
  double2* r = cfft_smem_t<1>(sa, sb, R.px, R.WMx);
  if (r != dst) {
    for (int j = threadIdx.x; j < L; j += blockDim.x) dst[j] = r[j];
  }
  __syncthreads();
}

// forward x transform of a packed real row held in `row` (destroyed) into dst[k], k < Kx
__device__ void row_r2c(double2* row, double2* scratch, double2* dst, const KMember& m, const KRes& R, double s0,
                        double s) {
  const int Kx = m.Kx, L = m.L;
  double2* z = cfft_smem_t<-1>(row, scratch, R.px, R.WMx);
  r2c_post2(z, [&](int k, double2 v) {  // v = 2 X_k
    const double f = 0.5 * (k == 0 ? s0 : s);
    double2 o = make_double2(v.x * f, v.y * f);
    if (k == 0) o.y = 0.0;
    dst[k] = o;
  }, Kx, L, R.WMx);
  __syncthreads();
}

// Inverse x transforms of nf mixed rows at once (weights 1): spectrum f (Kx entries from src(f))
// is staged in base + (2f+1) L, its packed spectrum built in base + 2f L, and the nf FFTs share
// their passes (more butterflies per pass than threads in one row's, one barrier per pass for
// all).  Returns the slot of field 0's packed grid row; field f's is 2 f L further.
template <class Src>
__device__ double2* rows_c2r_sets(double2* base, int nf, Src src, const KMember& m, const KRes& R) {
  const int Kx = m.Kx, L = m.L;
  for (int idx = threadIdx.x; idx < nf * Kx; idx += blockDim.x) {
    const int f = idx / Kx, k = idx - f * Kx;
    base[(2 * f + 1) * L + k] = ldcg2(&src(f)[k]);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nf * L; idx += blockDim.x) {
    const int f = idx / L, k = idx - f * L;
    const double2* S = base + (2 * f + 1) * L;
    base[2 * f * L + k] = c2r_entry<true>([&](int i) { return S[i]; }, k, Kx, L, R.WMx, 1.0, 1.0);
  }
  __syncthreads();
  cfft_smem_sets<1>(base, base + L, 2 * L, nf, R.px, 1);
  return (R.px.nrad & 1) ? base + L : base;
}

// Forward x transforms of nf packed grid rows at once: row f at a + 2 f L (destroyed), scratch at
// b + 2 f L; put(f, k, 2 X_k) for k < Kx (the unpacking's 1/2 is left to put).
template <class Put>
__device__ void rows_r2c_sets(double2* a, double2* b, int nf, Put put, const KMember& m, const KRes& R) {
  const int Kx = m.Kx, L = m.L;
  cfft_smem_sets<-1>(a, b, 2 * L, nf, R.px, 1);
  const double2* z = (R.px.nrad & 1) ? b : a;
  for (int idx = threadIdx.x; idx < nf * Kx; idx += blockDim.x) {
    const int f = idx / Kx, k = idx - f * Kx;
    const double2* Z = z + 2 * f * L;
    put(f, k, r2c_combine2(Z[k], cconj(Z[k == 0 ? 0 : L - k]), __ldg(&R.WMx[k])));
  }
  __syncthreads();
}

// ---- forward B tile ---------------------------------------------------------------------------
__device__ void b_forward(const KolArgs& A, const KMember& m, int tile) {
  extern __shared__ double2 ks[];
  const int Kx = m.Kx, M = m.M, L = m.L;
  const KRes& R = A.res[m.res];
  // ks[0, 8L): four transform sets (field f: slots 2f, 2f+1 of L entries); ks[8L, 8L+Kx): staging
  double2* st = ks + 8 * L;
  const int j0 = tile * A.RW, j1 = min(M, j0 + A.RW);
  const double invM = 1.0 / M;
  for (int j = j0; j < j1; ++j) {
    if (A.closure) {
      row_c2r(A.mixA[4] + m.off_mix + (long long)j * Kx, ks, ks, ks + L, st, m, R, 1.0, 1.0);
      double2* gw = reinterpret_cast<double2*>(A.gridW + m.off_grid + (long long)j * M);
      for (int i = threadIdx.x; i < L; i += blockDim.x) gw[i] = ks[i];
      __syncthreads();
    }
    double2 *prod = ks, *scratch = ks + L;
    if (A.nonlinear) {
      // u, v, w_x, w_y on the grid row, then u w_x + v w_y into the free slot of field 0
      const double2* r = rows_c2r_sets(ks, 4, [&](int f) { return A.mixA[f] + m.off_mix + (long long)j * Kx; }, m, R);
      prod = (r == ks) ? ks + L : ks;
      scratch = prod + 2 * L;
      for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const double2 u = r[i], v = r[2 * L + i], wx = r[4 * L + i], wy = r[6 * L + i];
        prod[i] = make_double2(fma(u.x, wx.x, v.x * wy.x), fma(u.y, wx.y, v.y * wy.y));
      }
    } else {
      for (int i = threadIdx.x; i < L; i += blockDim.x) prod[i] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    row_r2c(prod, scratch, A.mixB[0] + m.off_mix + (long long)j * Kx, m, R, invM, invM);
  }
}

// ---- adjoint C'A' tile ------------------------------------------------------------------------
// first: the first half (finish the VJP at X_n, inject the cotangent, solve for Y_n); otherwise Y_n is
// read from the Y ring.  second: the second half (W_{n-1} and the fields of X_{n-1} for the next VJP).
__device__ void ca_adjoint(const KolArgs& A, const KMember& m, int tile, int n, bool first, bool second) {
  extern __shared__ double2 ks[];
  const int N = m.N, Kx = m.Kx, M = m.M;
  const KRes& R = A.res[m.res];
  // The VJP's forward y transforms run two at a time (sets at ks + 2 p M, scratch + M) when the
  // accumulator lam fits beside them; otherwise one at a time in ks[0, 2M).
  const bool pairs = 4 * M + N <= A.smem_entries;
  double2* ca = ks;                             // M
  double2* cb = ca + M;                         // M
  double2* lam = pairs ? ks + 4 * M : cb + M;   // N
  double2* yc = pairs ? ks + 2 * M : lam + N;   // N (used after the VJP)
  const int kx0 = tile * A.CW, kx1 = min(Kx, kx0 + A.CW);
  const long long S = A.state_size;
  const int SN = A.S;
  for (int kx = kx0; kx < kx1; ++kx) {
    const long long col = m.off_state + (long long)kx * N;
    if (!first) {  // Y_n from the ring (computed by the previous launch)
      for (int q = threadIdx.x; q < N; q += blockDim.x) yc[q] = ldcg2(&A.Yr[n & 1][col + q]);
      __syncthreads();
    } else {
    for (int q = threadIdx.x; q < N; q += blockDim.x) lam[q] = make_double2(0.0, 0.0);
    __syncthreads();
    if (n < SN && (A.nonlinear || A.closure)) {
      // VJP: B_y^dagger of the grid cotangents, then the adjoint multipliers (identity for the
      // closure's input field)
      const int fa = A.nonlinear ? 0 : 4, fb = A.closure ? 5 : 4, per = pairs ? 2 : 1;
      for (int f0 = fa; f0 < fb; f0 += per) {
        const int np = min(per, fb - f0);
        for (int i = threadIdx.x; i < np * M; i += blockDim.x) {
          const int pq = i / M, j = i - pq * M;
          ks[pq * 2 * M + j] = ldcg2(&A.mixB[f0 + pq][m.off_mix + (long long)j * Kx + kx]);
        }
        __syncthreads();
        cfft_smem_sets<-1>(ks, ks + M, 2 * M, np, R.py, 1);
        const double2* r = (R.py.nrad & 1) ? ks + M : ks;
        for (int q = threadIdx.x; q < N; q += blockDim.x) {
          const int idx = yidx(q, N, M);
          if (idx < 0) continue;
          double2 l = lam[q];
          for (int pq = 0; pq < np; ++pq) {
            const int f = f0 + pq;
            const double2 v = r[pq * 2 * M + idx];
            if (f == 4) {
              l.x += v.x;
              l.y += v.y;
              continue;
            }
            // adjoint of i*s is -i*s: fmult with the negated multiplier
            const double2 fv = fmult(f, (double)kx, (double)kyof(q, N), v);
            l.x -= fv.x;
            l.y -= fv.y;
          }
          lam[q] = l;
        }
        __syncthreads();
      }
    }
    const int si = A.seed_at ? A.seed_at[n] : -1;
    const Coef c1 = (n + 1 <= SN) ? kcoef(n + 1, A.kc) : Coef{0, 0, 0, 0, 0};
    const Coef c2 = (n + 2 <= SN) ? kcoef(n + 2, A.kc) : Coef{0, 0, 0, 0, 0};
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
      double2 l = lam[q];
      if (si >= 0) {
        const double2 sd = A.seeds[(long long)si * S + col + q];
        l.x += sd.x; l.y += sd.y;
      }
      if (n + 1 <= SN) {
        const double2 y1 = ldcg2(&A.Yr[(n + 1) & 1][col + q]);
        l.x -= c1.a1 * y1.x; l.y -= c1.a1 * y1.y;
      }
      if (n + 2 <= SN) {
        const double2 y2 = ldcg2(&A.Yr[n & 1][col + q]);
        l.x -= c2.a2 * y2.x; l.y -= c2.a2 * y2.y;
      }
      lam[q] = l;
    }
    __syncthreads();
    if (n == 0) {
      for (int q = threadIdx.x; q < N; q += blockDim.x) A.out[col + q] = lam[q];
      __syncthreads();
      continue;
    }
    project_col(lam, N, kx);
    const Coef cn = kcoef(n, A.kc);
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
      const double ky = kyof(q, N);
      const double inv = 1.0 / (cn.a0 + ((double)kx * kx + ky * ky) * A.invRe);
      yc[q] = make_double2(lam[q].x * inv, lam[q].y * inv);
    }
    __syncthreads();
    }  // first half
    if (!second) {  // the launch ends at Y_n: store it for the next launch
      for (int q = threadIdx.x; q < N; q += blockDim.x) A.Yr[n & 1][col + q] = yc[q];
      __syncthreads();
      continue;
    }
    // W_{n-1} = c1^n Y_n + c2^{n+1} Y_{n+1}, read Y_{n+1} before Y_n overwrites Y_{n+2}
    const Coef cw1 = kcoef(n, A.kc);
    const Coef cw2 = (n + 1 <= SN) ? kcoef(n + 1, A.kc) : Coef{0, 0, 0, 0, 0};
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
      double2 w = make_double2(cw1.c1 * yc[q].x, cw1.c1 * yc[q].y);
      if (n + 1 <= SN) {
        const double2 y1 = ldcg2(&A.Yr[(n + 1) & 1][col + q]);
        w.x += cw2.c2 * y1.x; w.y += cw2.c2 * y1.y;
      }
      lam[q] = w;
      A.Yr[n & 1][col + q] = yc[q];
    }
    __syncthreads();
    if (!A.nonlinear && !A.closure) continue;
    // T_y^dagger W (inverse FFT with 1/M) -> mixA[4]
    for (int j = threadIdx.x; j < M; j += blockDim.x) ca[j] = make_double2(0.0, 0.0);
    __syncthreads();
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
      const int idx = yidx(q, N, M);
      if (idx >= 0) ca[idx] = lam[q];
    }
    {
      double2* r = col_fft<1>(ca, cb, R);
      const double invM = 1.0 / M;
      for (int j = threadIdx.x; j < M; j += blockDim.x)
        A.mixA[4][m.off_mix + (long long)j * Kx + kx] = make_double2(r[j].x * invM, r[j].y * invM);
    }
    // fields of X_{n-1} from the trajectory, their inverse y transforms two at a time (sets at
    // ks + 2 p M, scratch + M; 4M <= the CTA's shared memory for every member)
    const double2* xs = A.traj + (long long)(n - 1 - A.lo) * S + col;
    const int fa = A.nonlinear ? 0 : 4, fb = A.closure ? 5 : 4;
    for (int f0 = fa; f0 < fb; f0 += 2) {
      const int np = min(2, fb - f0);
      __syncthreads();
      for (int i = threadIdx.x; i < np * M; i += blockDim.x) {
        const int pq = i / M;
        ks[pq * 2 * M + (i - pq * M)] = make_double2(0.0, 0.0);
      }
      __syncthreads();
      for (int i = threadIdx.x; i < np * N; i += blockDim.x) {
        const int pq = i / N, q = i - pq * N, f = f0 + pq;
        const int idx = yidx(q, N, M);
        if (idx < 0) continue;
        const double2 x = ldcg2(&xs[q]);
        ks[pq * 2 * M + idx] = f < 4 ? fmult(f, (double)kx, (double)kyof(q, N), x) : x;
      }
      __syncthreads();
      cfft_smem_sets<1>(ks, ks + M, 2 * M, np, R.py, 1);
      const double2* r = (R.py.nrad & 1) ? ks + M : ks;
      for (int i = threadIdx.x; i < np * M; i += blockDim.x) {
        const int pq = i / M, j = i - pq * M, f = f0 + pq;
        // the closure's input field goes to slot 5 (slot 4 holds T^dagger W)
        A.mixA[f < 4 ? f : 5][m.off_mix + (long long)j * Kx + kx] = r[pq * 2 * M + j];
      }
    }
    __syncthreads();
  }
}

// ---- adjoint B' tile --------------------------------------------------------------------------
__device__ void b_adjoint(const KolArgs& A, const KMember& m, int tile) {
  extern __shared__ double2 ks[];
  const int Kx = m.Kx, M = m.M, L = m.L;
  const KRes& R = A.res[m.res];
  // ks[0, 8L): four transform sets (field f: slots 2f, 2f+1 of L entries); ks[8L, 8L+Kx): staging
  double2* st = ks + 8 * L;
  const int j0 = tile * A.RW, j1 = min(M, j0 + A.RW);
  for (int j = j0; j < j1; ++j) {
    if (!A.nonlinear) {  // closure only: omega and the grid cotangent g, for the CNN's backward pass
      if (A.closure) {
        row_c2r(A.mixA[4] + m.off_mix + (long long)j * Kx, ks, ks, ks + L, st, m, R, 1.0 / M, 0.5 / M);
        row_c2r(A.mixA[5] + m.off_mix + (long long)j * Kx, ks + 2 * L, ks + 2 * L, ks + 3 * L, st, m, R, 1.0, 1.0);
        double2* gw = reinterpret_cast<double2*>(A.gridW + m.off_grid + (long long)j * M);
        double2* gg = reinterpret_cast<double2*>(A.gridG + m.off_grid + (long long)j * M);
        for (int i = threadIdx.x; i < L; i += blockDim.x) { gw[i] = ks[2 * L + i]; gg[i] = ks[i]; }
        __syncthreads();
      }
      continue;
    }
    // u, v, w_x, w_y in one set of transforms; the free slots F_f = fr + 2 f L take g (F_0, with
    // F_1 as its scratch), the closure's omega (F_2, scratch F_3), then serve as the forward
    // transforms' scratch
    double2* r = rows_c2r_sets(ks, 4, [&](int f) { return A.mixA[f] + m.off_mix + (long long)j * Kx; }, m, R);
    double2* fr = (r == ks) ? ks + L : ks;
    row_c2r(A.mixA[4] + m.off_mix + (long long)j * Kx, fr, fr, fr + 2 * L, st, m, R, 1.0 / M, 0.5 / M);
    if (A.closure) {
      row_c2r(A.mixA[5] + m.off_mix + (long long)j * Kx, fr + 4 * L, fr + 4 * L, fr + 6 * L, st, m, R, 1.0, 1.0);
      double2* gw = reinterpret_cast<double2*>(A.gridW + m.off_grid + (long long)j * M);
      double2* gg = reinterpret_cast<double2*>(A.gridG + m.off_grid + (long long)j * M);
      for (int i = threadIdx.x; i < L; i += blockDim.x) { gw[i] = fr[4 * L + i]; gg[i] = fr[i]; }
      __syncthreads();
    }
    // grid cotangents of u, v, w_x, w_y: -g w_x, -g w_y, -g u, -g v
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
      const double2 u = r[i], v = r[2 * L + i], wx = r[4 * L + i], wy = r[6 * L + i], g = fr[i];
      r[i] = make_double2(-g.x * wx.x, -g.y * wx.y);
      r[2 * L + i] = make_double2(-g.x * wy.x, -g.y * wy.y);
      r[4 * L + i] = make_double2(-g.x * u.x, -g.y * u.y);
      r[6 * L + i] = make_double2(-g.x * v.x, -g.y * v.y);
    }
    __syncthreads();
    rows_r2c_sets(r, fr, 4, [&](int f, int k, double2 v) {  // v = 2 X_k; scales 1 (k = 0), 2
      const double sc = k == 0 ? 0.5 : 1.0;
      double2 o = make_double2(v.x * sc, v.y * sc);
      if (k == 0) o.y = 0.0;
      A.mixB[f][m.off_mix + (long long)j * Kx + k] = o;
    }, m, R);
  }
}

// ---- drivers ---------------------------------------------------------------------------------
__device__ __forceinline__ int find_member(const KolArgs& A, int r, bool ca) {
  int b = 0;
  for (int i = 0; i < A.nmem; ++i) {
    const int st = ca ? A.mem[i].caStart : A.mem[i].bStart;
    if (st <= r) b = i;
  }
  return b;
}

__device__ void run_item(const KolArgs& A, int stage, bool isCA, int b, int tile) {
  const KMember& m = A.mem[b];
  if (!A.adjoint) {
    if (isCA) ca_forward(A, m, tile, stage);
    else b_forward(A, m, tile);
  } else {
    const int n = A.n0 - stage;
    if (isCA) ca_adjoint(A, m, tile, n, !(A.prologue && stage == 0), !(A.lo > 0 && n == A.lo));
    else b_adjoint(A, m, tile);
  }
}

// bounded wait by thread 0 for *ctr >= target; false if the launch is being abandoned
__device__ bool wait_ge(int* ctr, int target, int* err, unsigned limit) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    unsigned it = 0;
    while (true) {
      if (*(volatile int*)ctr >= target) break;
      if (*(volatile int*)err) { ok = 0; break; }
      if (++it > limit) {
        atomicCAS(err, 0, 1);
        ok = 0;
        break;
      }
      __nanosleep(128);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__global__ void __launch_bounds__(kKolThreads) kol_persistent(const __grid_constant__ KolArgs A) {
  __shared__ int item;
  const int per = A.nCAtot + A.nBtot;
  const int nrun = A.nrun > 0 ? A.nrun : A.nstage;
  const int total = nrun * per - (A.stage0 + nrun == A.nstage ? A.nBtot : 0);  // the last stage has no B phase
  while (true) {
    if (threadIdx.x == 0) item = (*(volatile int*)A.err) ? total : atomicAdd(A.queue, 1);
    __syncthreads();
    const int it = item;
    __syncthreads();
    if (it >= total) break;
    const int stage = A.stage0 + it / per, r = it % per;
    const bool isCA = r < A.nCAtot;
    const int rr = isCA ? r : r - A.nCAtot;
    const int b = find_member(A, rr, isCA);
    const KMember& m = A.mem[b];
    const int tile = rr - (isCA ? m.caStart : m.bStart);
    const bool ok = isCA ? (stage == 0 || wait_ge(&A.bDone[b], stage * m.nB, A.err, A.spin_limit))
                         : wait_ge(&A.caDone[b], (stage + 1) * m.nCA, A.err, A.spin_limit);
    if (!ok) break;
    run_item(A, stage, isCA, b, tile);
    __syncthreads();
    if (threadIdx.x == 0 && b != A.drop_signal_member) {
      __threadfence();
      atomicAdd(isCA ? &A.caDone[b] : &A.bDone[b], 1);
    }
  }
}

// one phase of one stage as an ordinary launch (grid = tiles of all members)
__global__ void __launch_bounds__(kKolThreads) kol_phase(const __grid_constant__ KolArgs A, int stage, int isCA) {
  const int r = blockIdx.x;
  const int b = find_member(A, r, isCA != 0);
  const KMember& m = A.mem[b];
  const int tile = r - (isCA ? m.caStart : m.bStart);
  run_item(A, stage, isCA != 0, b, tile);
}

// x-forward transform of grid rows of the closure: mode 0 mixB[0] -= T_x(corr row) (the
// closure term enters F = -P + C with P stored), mode 1 mixB[4] = B_x^dagger(grid row).
__global__ void __launch_bounds__(kKolThreads) closure_rows_kernel(const __grid_constant__ KolArgs A, const double* grid,
                                                                  int mode) {
  extern __shared__ double2 ks[];
  const int b = blockIdx.y;
  const KMember& m = A.mem[b];
  const int j = blockIdx.x;
  if (j >= m.M) return;
  const KRes& R = A.res[m.res];
  const int L = m.L, Kx = m.Kx;
  double2* sa = ks;
  double2* sb = sa + L;
  double2* st = sb + L;
  const double2* g = reinterpret_cast<const double2*>(grid + m.off_grid + (long long)j * m.M);
  for (int i = threadIdx.x; i < L; i += blockDim.x) sa[i] = g[i];
  __syncthreads();
  if (mode == 0) {
    row_r2c(sa, sb, st, m, R, 1.0 / m.M, 1.0 / m.M);
    double2* dst = A.mixB[0] + m.off_mix + (long long)j * Kx;
    for (int k = threadIdx.x; k < Kx; k += blockDim.x) {
      const double2 v = dst[k];
      dst[k] = make_double2(v.x - st[k].x, v.y - st[k].y);
    }
  } else {
    row_r2c(sa, sb, A.mixB[4] + m.off_mix + (long long)j * Kx, m, R, 1.0, 2.0);
  }
}

// 4D-Var misfit per (member, observation) and its cotangent seeds[m] = H^T H (X_{n_m} - obs_m)
__global__ void fourdvar_kernel(const KMember* mem, const double2* traj, const int* obs_steps, const double2* obs,
                                long long S, int kmax, double2* seeds, double* partial, int n_obs) {
  const int b = blockIdx.x, o = blockIdx.y;
  const KMember m = mem[b];
  const double2* X = traj + (long long)obs_steps[o] * S + m.off_state;
  const double2* Ob = obs + (long long)o * S + m.off_state;
  double2* sd = seeds + (long long)o * S + m.off_state;
  double acc = 0.0;
  const int n = m.Kx * m.N;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int kx = i / m.N, q = i % m.N;
    const int ky = kyof(q, m.N);
    const bool keep = kx <= kmax && (ky <= kmax && ky >= -kmax);
    double2 d = make_double2(0.0, 0.0);
    if (keep) {
      const double2 x = X[i], y = Ob[i];
      d = make_double2(x.x - y.x, x.y - y.y);
      acc += d.x * d.x + d.y * d.y;
    }
    sd[i] = d;
  }
  __shared__ double red[kKolThreads];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(long long)b * n_obs + o] = 0.5 * red[0];
}

__global__ void sum_rows_kernel(const double* partial, int n_obs, int nmem, double* J) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nmem) return;
  double s = 0.0;
  for (int o = 0; o < n_obs; ++o) s += partial[(long long)b * n_obs + o];
  J[b] = s;
}

// y += x (n values)
__global__ void add_kernel(double* __restrict__ y, const double* __restrict__ x, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] += x[i];
}

// ---- training support for the learned closure -------------------------------------------------
// Spectral truncation of B fine members (Nf modes, layout [kx][ky] of SPADJ_KOLMOGOROV2D) to Nc
// modes: coarse (kx, ky) = fine (kx, ky) for kx < Nc/2 and |ky| < Nc/2; the coarse ky = -Nc/2 row
// is zero (the layout holds it at zero).
__global__ void restrict_kernel(const double2* __restrict__ fine, int Nf, int Nc, int B, double2* __restrict__ coarse) {
  const int Kc = Nc / 2, Kf = Nf / 2;
  const long long per_c = (long long)Kc * Nc, n = per_c * B;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / per_c);
    const int r = (int)(i - (long long)b * per_c);
    const int kx = r / Nc, j = r - kx * Nc;
    double2 v = make_double2(0.0, 0.0);
    if (j != Nc / 2) {
      const int ky = j < Nc / 2 ? j : j - Nc;
      const int jf = ky >= 0 ? ky : Nf + ky;
      v = fine[(long long)b * Kf * Nf + (long long)kx * Nf + jf];
    }
    coarse[i] = v;
  }
}

// One Adam step (Kingma & Ba 2015) on n parameters: m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
// p <- p - lr mhat / (sqrt(vhat) + eps) with the bias corrections c1 = 1 - b1^t, c2 = 1 - b2^t.
__global__ void adam_kernel(int n, const double* __restrict__ g, double b1, double b2, double lr, double eps, double c1,
                            double c2, double* __restrict__ m, double* __restrict__ v, double* __restrict__ p) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double gi = g[i];
    const double mi = b1 * m[i] + (1.0 - b1) * gi;
    const double vi = b2 * v[i] + (1.0 - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrt(vi / c2) + eps);
  }
}

// ---- host ------------------------------------------------------------------------------------

bool fft_len_ok(int n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

struct Kol : EqImpl {
  std::vector<KMember> hm;
  std::vector<int> resN;
  int nmem = 0;
  long long state_size = 0, mix_size = 0, grid_size = 0;
  int closure = 0;
  DevBuf gridW, gridG, corr, xq, hbuf[3], dact[3], dh, dz, dz2, pbuf, wq, bq, part, gp, chunkbuf;
  static constexpr int kWgradChunks = 8;
  int Lmax = 0, Mmax = 0, Nmax = 0, Kxmax = 0;
  double Re = 100.0, dt = 0;
  int forcing = 1, nonlinear = 1;
  int CW = 4, RW = 2, ctas_per_sm = 0, persistent = 1;
  unsigned spin_limit = kSpinLimit;
  int drop_signal_member = -1;
  DevBuf dmem, tables, Xr[2], Fr[2], Yr[2], mixA, mixB, ctr, trajbuf, seedbuf, seedmap, obsbuf, obsteps, partial, Jd,
      tmp;
  int n_obs = 0, obs_kmax = 32;
  std::vector<int> obs_steps_h;
  KRes kres[kMaxRes];
  size_t smem = 0;
  int grid_persistent = 0;

  size_t state_len(int which) const override {
    if (which == 0 || which == 3) return (size_t)(2 * state_size);
    if (which == 1) {
      size_t g = 0;
      for (auto& m : hm) g += (size_t)m.M * m.M;
      return g;
    }
    if (which == 2) return closure ? (size_t)cnn::n_params() : 0;
    return 0;
  }

  void layout() {
    int ca = 0, bb = 0;
    for (auto& m : hm) {
      m.nCA = (m.Kx + CW - 1) / CW;
      m.nB = (m.M + RW - 1) / RW;
      m.caStart = ca;
      m.bStart = bb;
      ca += m.nCA;
      bb += m.nB;
    }
  }
  int nCAtot() const { return hm.empty() ? 0 : hm.back().caStart + hm.back().nCA; }
  int nBtot() const { return hm.empty() ? 0 : hm.back().bStart + hm.back().nB; }

  spadj_status init(Problem* p) {
    const spadj_desc& d = p->desc;
    if (d.scheme != SPADJ_SBDF1 && d.scheme != SPADJ_SBDF2)
      return p->fail(SPADJ_ERR_UNSUPPORTED, "kolmogorov: scheme must be SBDF2");
    nmem = d.batch;
    Re = d.params[0];
    if (!(Re > 0)) return p->fail(SPADJ_ERR_INVALID, "kolmogorov: params[0] (Reynolds number) must be > 0");
    forcing = d.params[1] == 1.0 ? 0 : 1;
    nonlinear = d.nonlinear;
    dt = d.dt;
    long long offs = 0, offm = 0, offg = 0;
    closure = d.closure ? 1 : 0;
    for (int b = 0; b < nmem; ++b) {
      const int N = d.batch_n ? d.batch_n[b] : d.n[0];
      if (N < 8 || N % 4 != 0 || !fft_len_ok(3 * N / 2) || N > 1024)
        return p->fail(SPADJ_ERR_INVALID, "kolmogorov: each resolution must be a multiple of 4 in 8..1024 with 3N/2 = 2^a 3^b");
      int r = -1;
      for (size_t i = 0; i < resN.size(); ++i)
        if (resN[i] == N) r = (int)i;
      if (r < 0) {
        if ((int)resN.size() >= kMaxRes) return p->fail(SPADJ_ERR_UNSUPPORTED, "kolmogorov: at most 4 distinct resolutions");
        resN.push_back(N);
        r = (int)resN.size() - 1;
      }
      KMember m{};
      m.N = N; m.Kx = N / 2; m.M = 3 * N / 2; m.L = m.M / 2; m.res = r;
      m.off_state = offs; m.off_mix = offm; m.off_grid = offg;
      offs += (long long)m.Kx * N;
      offm += (long long)m.M * m.Kx;
      offg += (long long)m.M * m.M;
      if (closure && b > 0 && N != hm[0].N)
        return p->fail(SPADJ_ERR_UNSUPPORTED, "kolmogorov: the learned closure needs one resolution for the whole batch");
      hm.push_back(m);
      Lmax = std::max(Lmax, m.L); Mmax = std::max(Mmax, m.M); Nmax = std::max(Nmax, N); Kxmax = std::max(Kxmax, m.Kx);
    }
    state_size = offs;
    mix_size = offm;
    grid_size = offg;
    // twiddle tables per resolution: WMx (M entries) then W2M (2M entries)
    std::vector<double2> ht;
    std::vector<size_t> toff, soff;
    for (size_t i = 0; i < resN.size(); ++i) {
      const int M = 3 * resN[i] / 2;
      kres[i].px = make_plan(M / 2);
      kres[i].py = make_plan(M);
    }
    for (size_t i = 0; i < resN.size(); ++i) {
      const int N = resN[i];
      const int M = 3 * N / 2;
      toff.push_back(ht.size());
      for (int m = 0; m < M; ++m) {
        const double th = -2.0 * M_PI * m / M;
        ht.push_back(make_double2(std::cos(th), std::sin(th)));
      }
      for (int m = 0; m < 2 * M; ++m) {
        const double th = -2.0 * M_PI * m / (2.0 * M);
        ht.push_back(make_double2(std::cos(th), std::sin(th)));
      }
      // the butterflies' scaled-twiddle records of the x and y plans
      soff.push_back(ht.size());
      const std::vector<double2> sx = scaled_twiddle_table(kres[i].px);
      ht.insert(ht.end(), sx.begin(), sx.end());
      soff.push_back(ht.size());
      const std::vector<double2> sy = scaled_twiddle_table(kres[i].py);
      ht.insert(ht.end(), sy.begin(), sy.end());
    }
    SPADJ_CUDA_TRY(p, tables.ensure(sizeof(double2) * ht.size()));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(tables.ptr, ht.data(), sizeof(double2) * ht.size(), cudaMemcpyHostToDevice, p->stream));
    for (size_t i = 0; i < resN.size(); ++i) {
      const int M = 3 * resN[i] / 2;
      kres[i].WMx = tables.as<double2>() + toff[i];
      kres[i].W2M = tables.as<double2>() + toff[i] + M;
      bind_scaled_twiddles(kres[i].px, tables.as<double2>() + soff[2 * i]);
      bind_scaled_twiddles(kres[i].py, tables.as<double2>() + soff[2 * i + 1]);
    }
    const size_t sb = sizeof(double2) * state_size, mb = sizeof(double2) * mix_size;
    for (int i = 0; i < 2; ++i) {
      SPADJ_CUDA_TRY(p, Xr[i].ensure(sb));
      SPADJ_CUDA_TRY(p, Fr[i].ensure(sb));
      SPADJ_CUDA_TRY(p, Yr[i].ensure(sb));
    }
    SPADJ_CUDA_TRY(p, mixA.ensure(6 * mb));
    SPADJ_CUDA_TRY(p, mixB.ensure(5 * mb));
    if (closure) {
      // The CNN needs whole-member grids between the steps, so the persistent scheduler runs one
      // launch per step.  It pays off only when the batch has enough grid rows to keep every CTA
      // busy while the members' row tiles wait on their column tiles; measured with 64-mode
      // windows (forward sweep, us per window-step, per-step persistent with 4 rows per row tile
      // against one launch per phase with 2): 128 windows 7.8 against 8.1 (training iteration
      // 57.3 against 59.8 ms), 64 windows 9.4 against 8.9, 16 windows 19.1 against 15.4.  Hence:
      // at least 64 grid rows per SM -> per-step persistent launches with 4 rows per row tile,
      // else one launch per phase with 2 (option 0 overrides the launch form).
      {
        int dev = 0, sms = 0;
        SPADJ_CUDA_TRY(p, cudaGetDevice(&dev));
        SPADJ_CUDA_TRY(p, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        long long rows = 0;
        for (auto& m : hm) rows += m.M;
        persistent = rows >= 64LL * sms ? 1 : 0;
        RW = persistent ? 4 : 2;
      }
      const size_t gb = sizeof(double) * grid_size;
      const size_t np = (size_t)cnn::n_params();
      const size_t act = (size_t)grid_size * cnn::kHid;
      SPADJ_CUDA_TRY(p, gridW.ensure(gb));
      SPADJ_CUDA_TRY(p, gridG.ensure(gb));
      SPADJ_CUDA_TRY(p, corr.ensure(gb));
      SPADJ_CUDA_TRY(p, xq.ensure(sizeof(__nv_bfloat16) * grid_size));
      for (int l = 0; l < 3; ++l) {
        SPADJ_CUDA_TRY(p, hbuf[l].ensure(sizeof(__nv_bfloat16) * act));
        SPADJ_CUDA_TRY(p, dact[l].ensure(sizeof(float) * act));
      }
      SPADJ_CUDA_TRY(p, dh.ensure(sizeof(float) * act));
      SPADJ_CUDA_TRY(p, dz.ensure(sizeof(__nv_bfloat16) * act));
      SPADJ_CUDA_TRY(p, dz2.ensure(sizeof(__nv_bfloat16) * act));
      SPADJ_CUDA_TRY(p, pbuf.ensure(sizeof(double) * np));
      SPADJ_CUDA_TRY(p, wq.ensure(sizeof(__nv_bfloat16) * np));
      SPADJ_CUDA_TRY(p, bq.ensure(sizeof(float) * np));
      SPADJ_CUDA_TRY(p, part.ensure(sizeof(float) * np * nmem));
      SPADJ_CUDA_TRY(p, gp.ensure(sizeof(double) * np));
      // weight partials [member][tap][chunk][32 x 32], then the bias partials [member][chunk][32]
      SPADJ_CUDA_TRY(p, chunkbuf.ensure(sizeof(float) * (size_t)nmem * kWgradChunks * (9 * 1024 + 32)));
      SPADJ_CUDA_TRY(p, cnnerr.ensure(sizeof(int)));
      SPADJ_CUDA_TRY(p, cudaMemsetAsync(cnnerr.ptr, 0, sizeof(int), p->stream));
      {
        int dev = 0;
        SPADJ_CUDA_TRY(p, cudaGetDevice(&dev));
        SPADJ_CUDA_TRY(p, cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev));
      }
      SPADJ_CUDA_TRY(p, cudaFuncSetAttribute(cnn::conv32_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)cnn::kTcSmem));
      // the halo-staged forms need two staging buffers of the grid's halo range: up to a 764-point
      // grid they fit one CTA; larger grids use the per-tap forms
      halo_fits = cnn::wgrad_halo_smem(hm[0].M) <= kHaloSmemMax && cnn::halo_smem(hm[0].M) <= kHaloSmemMax;
      if (halo_fits) {
        SPADJ_CUDA_TRY(p, cudaFuncSetAttribute(cnn::conv32_halo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)cnn::halo_smem(hm[0].M)));
        SPADJ_CUDA_TRY(p, cudaFuncSetAttribute(cnn::wgrad32_halo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)cnn::wgrad_halo_smem(hm[0].M)));
      }
      SPADJ_CUDA_TRY(p, cudaMemsetAsync(pbuf.ptr, 0, sizeof(double) * np, p->stream));
      cnn::convert_kernel<<<64, 256, 0, p->stream>>>(pbuf.as<double>(), wq.as<__nv_bfloat16>(), bq.as<float>());
      spadj_status st = check_launch(p, "closure convert");
      if (st != SPADJ_OK) return st;
    }
    SPADJ_CUDA_TRY(p, ctr.ensure(sizeof(int) * (2 * (size_t)nmem + 2)));
    SPADJ_CUDA_TRY(p, tmp.ensure(sb));
    // shared memory: max over tile kinds (B and B': 8 L + Kx, four transform sets and their
    // staging; CA': 2 M + 2 N, or 4 M + N with its VJP transforms in pairs).  The paired form's
    // size is taken when it keeps as many CTAs resident per SM.
    {
      const size_t base = sizeof(double2) * std::max<size_t>(8 * (size_t)Lmax + Kxmax, 2 * (size_t)Mmax + 2 * (size_t)Nmax);
      const size_t ext = std::max<size_t>(base, sizeof(double2) * (4 * (size_t)Mmax + Nmax));
      smem = base;
      if (ext > base && ext <= 227 * 1024) {
        int ob = 0, oe = 0;
        SPADJ_CUDA_TRY(p, cudaFuncSetAttribute(kol_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ext));
        SPADJ_CUDA_TRY(p, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ob, kol_persistent, kKolThreads, base));
        SPADJ_CUDA_TRY(p, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oe, kol_persistent, kKolThreads, ext));
        if (oe >= ob) smem = ext;
      }
    }
    SPADJ_CUDA_TRY(p, cudaFuncSetAttribute(kol_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SPADJ_CUDA_TRY(p, cudaFuncSetAttribute(kol_phase, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    layout();
    SPADJ_CUDA_TRY(p, dmem.ensure(sizeof(KMember) * nmem));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(dmem.ptr, hm.data(), sizeof(KMember) * nmem, cudaMemcpyHostToDevice, p->stream));
    SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    return SPADJ_OK;
  }

  spadj_status sync_members(Problem* p) {
    layout();
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(dmem.ptr, hm.data(), sizeof(KMember) * nmem, cudaMemcpyHostToDevice, p->stream));
    return SPADJ_OK;
  }

  KolArgs base_args() {
    KolArgs A{};
    A.nmem = nmem;
    A.mem = dmem.as<KMember>();
    for (int i = 0; i < kMaxRes; ++i) A.res[i] = kres[i];
    A.Re = Re; A.dt = dt; A.CW = CW; A.RW = RW;
    A.invRe = 1.0 / Re;
    const double kc[2][5] = {{1.0 / dt, -1.0 / dt, 0.0, 1.0, 0.0}, {1.5 / dt, -2.0 / dt, 0.5 / dt, 2.0, -1.0}};
    for (int r = 0; r < 2; ++r)
      for (int i = 0; i < 5; ++i) A.kc[r][i] = kc[r][i];
    A.nCAtot = nCAtot(); A.nBtot = nBtot();
    A.forcing = forcing; A.nonlinear = nonlinear;
    for (int i = 0; i < 2; ++i) { A.Xr[i] = Xr[i].as<double2>(); A.Fr[i] = Fr[i].as<double2>(); A.Yr[i] = Yr[i].as<double2>(); }
    for (int f = 0; f < 6; ++f) A.mixA[f] = mixA.as<double2>() + (size_t)f * mix_size;
    for (int f = 0; f < 5; ++f) A.mixB[f] = mixB.as<double2>() + (size_t)f * mix_size;
    A.closure = closure;
    A.gridW = gridW.as<double>();
    A.gridG = gridG.as<double>();
    A.state_size = state_size;
    int* c = ctr.as<int>();
    A.queue = c; A.err = c + 1; A.caDone = c + 2; A.bDone = c + 2 + nmem;
    A.spin_limit = spin_limit;
    A.smem_entries = (int)(smem / sizeof(double2));
    A.drop_signal_member = drop_signal_member;
    return A;
  }

  spadj_status launch(Problem* p, KolArgs& A) {
    const int per = A.nCAtot + A.nBtot;
    if (persistent) {
      cudaEvent_t t = closure ? nullptr : p->tic();
      SPADJ_CUDA_TRY(p, cudaMemsetAsync(ctr.ptr, 0, sizeof(int) * (2 * (size_t)nmem + 2), p->stream));
      if (!grid_persistent) {
        int dev = 0, sms = 0, occ = 0;
        SPADJ_CUDA_TRY(p, cudaGetDevice(&dev));
        SPADJ_CUDA_TRY(p, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        SPADJ_CUDA_TRY(p, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kol_persistent, kKolThreads, smem));
        if (occ < 1) return p->fail(SPADJ_ERR_INVALID, "kolmogorov: kernel does not fit on an SM");
        const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
        grid_persistent = sms * per_sm;
      }
      if (!closure) {
        kol_persistent<<<grid_persistent, kKolThreads, smem, p->stream>>>(A);
        spadj_status s = check_launch(p, "kolmogorov persistent");
        p->toc(t, KC_FUSED, work_flops(A));
        return s;
      }
      // closure: one persistent launch per step over that step's phases of all members (a member's
      // B tiles start as soon as its own CA tiles are done), the network passes between the launches
      const double per_stage = A.nstage > 1 ? work_flops(A) / (A.nstage - 1) : 0.0;
      for (int st = 0; st < A.nstage; ++st) {
        cudaEvent_t ts = p->tic();
        if (st > 0) SPADJ_CUDA_TRY(p, cudaMemsetAsync(ctr.ptr, 0, sizeof(int), p->stream));  // the item queue only
        A.stage0 = st;
        A.nrun = 1;
        kol_persistent<<<grid_persistent, kKolThreads, smem, p->stream>>>(A);
        spadj_status s = check_launch(p, "kolmogorov persistent step");
        if (s != SPADJ_OK) return s;
        p->toc(ts, KC_FUSED, st + 1 < A.nstage ? per_stage : 0.0);
        if (st + 1 < A.nstage) {
          s = A.adjoint ? closure_backward(p, A) : closure_forward(p, A);
          if (s != SPADJ_OK) return s;
        }
      }
      return SPADJ_OK;
    }
    // one launch per phase; the solver's phases and the closure's network passes are timed
    // separately (classes fused and cnn), stage by stage
    const double per_stage = A.nstage > 1 ? work_flops(A) / (A.nstage - 1) : 0.0;
    for (int st = 0; st < A.nstage; ++st) {
      cudaEvent_t ts = p->tic();
      kol_phase<<<A.nCAtot, kKolThreads, smem, p->stream>>>(A, st, 1);
      spadj_status s = check_launch(p, "kolmogorov phase CA");
      if (s != SPADJ_OK) return s;
      if (st + 1 < A.nstage) {
        kol_phase<<<A.nBtot, kKolThreads, smem, p->stream>>>(A, st, 0);
        if ((s = check_launch(p, "kolmogorov phase B")) != SPADJ_OK) return s;
      }
      p->toc(ts, KC_FUSED, st + 1 < A.nstage ? per_stage : 0.0);
      if (st + 1 < A.nstage && closure) {
        s = A.adjoint ? closure_backward(p, A) : closure_forward(p, A);
        if (s != SPADJ_OK) return s;
      }
    }
    (void)per;
    return SPADJ_OK;
  }

  // algorithmic FP64 flops of a launch: complex y-FFTs (5 M log2 M per column) and real
  // x-FFTs (2.5 M log2 M per row); forward stage: 5 y + 5 x, adjoint: 9 y + 9 x
  double work_flops(const KolArgs& A) const {
    double f = 0;
    const double ny = A.adjoint ? 9 : 5, nx = A.adjoint ? 9 : 5;
    for (auto& m : hm) {
      const double lg = std::log2((double)m.M);
      f += ny * m.Kx * 5.0 * m.M * lg + nx * m.M * 2.5 * m.M * lg;
    }
    return f * std::max(0, A.nstage - 1);
  }

  spadj_status check_err(Problem* p) {
    int e = 0;
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(&e, ctr.as<int>() + 1, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    if (e) return p->fail(SPADJ_ERR_TIMEOUT, "kolmogorov: a bounded wait in the persistent launch gave up");
    return SPADJ_OK;
  }

  spadj_status run_forward(Problem* p, int n_steps, const double* x0, double* x_out, double2* traj) {
    KolArgs A = base_args();
    A.adjoint = 0;
    A.nstage = n_steps + 1;
    A.S = n_steps;
    A.x0 = reinterpret_cast<const double2*>(x0);
    A.traj = traj;
    A.out = reinterpret_cast<double2*>(x_out);
    spadj_status s = launch(p, A);
    if (s != SPADJ_OK) return s;
    return persistent ? check_err(p) : SPADJ_OK;
  }

  spadj_status run_adjoint(Problem* p, int n_steps, double2* traj, const std::vector<int>& seed_at, const double2* seeds,
                           double* grad) {
    SPADJ_CUDA_TRY(p, seedmap.ensure(sizeof(int) * (n_steps + 1)));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(seedmap.ptr, seed_at.data(), sizeof(int) * (n_steps + 1), cudaMemcpyHostToDevice,
                                      p->stream));
    KolArgs A = base_args();
    A.adjoint = 1;
    A.nstage = n_steps + 1;
    A.S = n_steps;
    A.n0 = n_steps;
    A.traj = traj;
    A.out = reinterpret_cast<double2*>(grad);
    A.seed_at = seedmap.as<int>();
    A.seeds = seeds;
    spadj_status s = launch(p, A);
    if (s != SPADJ_OK) return s;
    return persistent ? check_err(p) : cudaStreamSynchronize(p->stream) == cudaSuccess ? SPADJ_OK
                                                                                       : p->fail(SPADJ_ERR_CUDA, "sync");
  }

  // ---- segments: checkpointed sweeps and the step entry points ----------------------------------
  // Restart state of step n (three states, the augmented state of the two-step scheme):
  // [X_n, X_{n-1}, F(X_{n-1})]; for n = 0 only X_0 is read.
  size_t sbytes() const { return sizeof(double2) * (size_t)state_size; }

  // k steps n0 -> n0 + k from the restart state rs (device); traj (nullable): X_{n0}..X_{n0+k};
  // x_out: X_{n0+k}; rs_out (nullable, may equal rs): the restart state of n0 + k
  spadj_status run_forward_seg(Problem* p, int n0, int k, const double2* rs, double2* traj, double2* x_out,
                               double2* rs_out) {
    const size_t sb = sbytes();
    const long long S = state_size;
    if (n0 >= 1) {
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(Xr[(n0 - 1) & 1].ptr, rs + S, sb, cudaMemcpyDeviceToDevice, p->stream));
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(Fr[(n0 - 1) & 1].ptr, rs + 2 * S, sb, cudaMemcpyDeviceToDevice, p->stream));
    }
    SPADJ_CUDA_TRY(p, segx0.ensure(sb));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(segx0.ptr, rs, sb, cudaMemcpyDeviceToDevice, p->stream));
    KolArgs A = base_args();
    A.adjoint = 0;
    A.nstage = k + 1;
    A.S = k;
    A.n0 = n0;
    A.x0 = segx0.as<double2>();
    A.traj = traj;
    A.out = x_out;
    spadj_status st = launch(p, A);
    if (st != SPADJ_OK) return st;
    if (persistent && (st = check_err(p)) != SPADJ_OK) return st;
    if (rs_out && k >= 1) {
      const int n1 = n0 + k;
      if (rs_out != x_out) SPADJ_CUDA_TRY(p, cudaMemcpyAsync(rs_out, x_out, sb, cudaMemcpyDeviceToDevice, p->stream));
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(rs_out + S, Xr[(n1 - 1) & 1].ptr, sb, cudaMemcpyDeviceToDevice, p->stream));
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(rs_out + 2 * S, Fr[(n1 - 1) & 1].ptr, sb, cudaMemcpyDeviceToDevice, p->stream));
    }
    return SPADJ_OK;
  }

  // adjoint indices hi .. lo of a horizon N over the segment trajectory seg = X_lo .. X_hi (prologue at
  // hi + 1 when hi < N: the adjoint variables Y_{hi+1}, Y_{hi+2} are in the Y ring); horizon = N for
  // the weights and the seed (or larger in step mode).  grad (nullable unless lo = 0) receives dJ/dX_0.
  spadj_status run_adjoint_seg(Problem* p, int N, int lo, int hi, const double2* seg, const int* seedmap_dev,
                               const double2* seeds, double* grad, int horizon) {
    KolArgs A = base_args();
    A.adjoint = 1;
    A.S = horizon;
    A.prologue = hi < N ? 1 : 0;
    A.n0 = hi + A.prologue;
    A.lo = lo;
    A.nstage = hi - lo + 1 + A.prologue;
    A.traj = const_cast<double2*>(seg);
    A.out = reinterpret_cast<double2*>(grad);
    A.seed_at = seedmap_dev;
    A.seeds = seeds;
    spadj_status st = launch(p, A);
    if (st != SPADJ_OK) return st;
    return persistent ? check_err(p) : SPADJ_OK;
  }

  // Checkpointed reverse sweep: H segments of K = ceil(N / H) steps; the restart state at each segment
  // start is kept (device slots, or page-locked host slots with host = true); each segment's
  // trajectory (K + 1 states) is recomputed before it is reversed, last segment first, and the
  // adjoint variables pass from one segment's launch to the next through the Y ring.  Observation
  // states (4D-Var) are kept from the first forward sweep.  seed_at[n] indexes seeds (device) for the
  // cotangent injected at X_n (objective_kind < 0), or the objective's seeds are formed here.
  DevBuf segx0, segbuf, rsbuf, cslots, obsstates, obsidx;
  HostBuf hcslots;
  spadj_status reverse_seg(Problem* p, const double* x0, int N, int H, bool host, bool objective,
                           const std::vector<int>& seed_at_in, const double2* seeds_in, double* grad, double* J_host) {
    H = std::max(1, std::min(H, N));
    const int K = (N + H - 1) / H;
    H = (N + K - 1) / K;
    const size_t sb = sbytes();
    const long long S = state_size;
    SPADJ_CUDA_TRY(p, segbuf.ensure(sb * (size_t)(K + 1)));
    SPADJ_CUDA_TRY(p, rsbuf.ensure(3 * sb));
    if (host) SPADJ_CUDA_TRY(p, hcslots.ensure(3 * sb * (size_t)H));
    else SPADJ_CUDA_TRY(p, cslots.ensure(3 * sb * (size_t)H));
    auto slot = [&](int j) {
      return host ? hcslots.as<char>() + (size_t)j * 3 * sb : cslots.as<char>() + (size_t)j * 3 * sb;
    };
    const cudaMemcpyKind to_slot = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind from_slot = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    double2* rs = rsbuf.as<double2>();
    double2* seg = segbuf.as<double2>();
    std::vector<int> seed_at = seed_at_in;
    const double2* seeds = seeds_in;
    if (objective) {
      SPADJ_CUDA_TRY(p, obsstates.ensure(sb * (size_t)n_obs));
      SPADJ_CUDA_TRY(p, obsidx.ensure(sizeof(int) * (size_t)n_obs));
      std::vector<int> idx(n_obs);
      for (int i = 0; i < n_obs; ++i) idx[i] = i;
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(obsidx.ptr, idx.data(), sizeof(int) * n_obs, cudaMemcpyHostToDevice, p->stream));
      SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    }
    // first forward sweep: segment starts into the slots, observation states kept
    SPADJ_CUDA_TRY(p, cudaMemsetAsync(rs, 0, 3 * sb, p->stream));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(rs, x0, sb, cudaMemcpyDeviceToDevice, p->stream));
    for (int j = 0; j < H; ++j) {
      const int a = j * K, b = std::min(N, a + K);
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(slot(j), rs, 3 * sb, to_slot, p->stream));
      spadj_status st = run_forward_seg(p, a, b - a, rs, objective ? seg : nullptr, tmp.as<double2>(), rs);
      if (st != SPADJ_OK) return st;
      if (objective)
        for (int i = 0; i < n_obs; ++i)
          if (obs_steps_h[i] > a && obs_steps_h[i] <= b)
            SPADJ_CUDA_TRY(p, cudaMemcpyAsync(obsstates.as<double2>() + (size_t)i * S, seg + (size_t)(obs_steps_h[i] - a) * S,
                                              sb, cudaMemcpyDeviceToDevice, p->stream));
    }
    if (objective) {
      SPADJ_CUDA_TRY(p, seedbuf.ensure(sb * (size_t)n_obs));
      SPADJ_CUDA_TRY(p, partial.ensure(sizeof(double) * (size_t)nmem * n_obs));
      SPADJ_CUDA_TRY(p, Jd.ensure(sizeof(double) * nmem));
      cudaEvent_t t = p->tic();
      fourdvar_kernel<<<dim3(nmem, n_obs), kKolThreads, 0, p->stream>>>(dmem.as<KMember>(), obsstates.as<double2>(),
                                                                        obsidx.as<int>(), obsbuf.as<double2>(), S,
                                                                        obs_kmax, seedbuf.as<double2>(),
                                                                        partial.as<double>(), n_obs);
      sum_rows_kernel<<<(nmem + 127) / 128, 128, 0, p->stream>>>(partial.as<double>(), n_obs, nmem, Jd.as<double>());
      p->toc(t, KC_OBJECTIVE, 4.0 * state_size * n_obs);
      spadj_status st = check_launch(p, "kolmogorov 4dvar");
      if (st != SPADJ_OK) return st;
      seed_at.assign(N + 1, -1);
      for (int i = 0; i < n_obs; ++i) seed_at[obs_steps_h[i]] = i;
      seeds = seedbuf.as<double2>();
    }
    SPADJ_CUDA_TRY(p, seedmap.ensure(sizeof(int) * (N + 1)));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(seedmap.ptr, seed_at.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, p->stream));
    // reverse, last segment first
    for (int j = H - 1; j >= 0; --j) {
      const int a = j * K, b = std::min(N, a + K);
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(rs, slot(j), 3 * sb, from_slot, p->stream));
      spadj_status st = run_forward_seg(p, a, b - a, rs, seg, tmp.as<double2>(), nullptr);
      if (st != SPADJ_OK) return st;
      const int hi = (b == N) ? N : b - 1;
      if ((st = run_adjoint_seg(p, N, a, hi, seg, seedmap.as<int>(), seeds, grad, N)) != SPADJ_OK) return st;
    }
    SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));  // host staging (seed map, host slots)
    if (objective && J_host) {
      SPADJ_CUDA_TRY(p, cudaMemcpy(J_host, Jd.ptr, sizeof(double) * nmem, cudaMemcpyDeviceToHost));
    }
    return SPADJ_OK;
  }

  int step_blocks(int which) const override { return which == 0 ? 3 : 2; }

  spadj_status step_forward(Problem* p, int n, const double* s_n, double* s_np1) override {
    if (n < 0) return p->fail(SPADJ_ERR_INVALID, "step: n < 0");
    SPADJ_CUDA_TRY(p, rsbuf.ensure(3 * sbytes()));
    SPADJ_CUDA_TRY(p, segbuf.ensure(2 * sbytes()));
    double2* out = reinterpret_cast<double2*>(s_np1);
    return run_forward_seg(p, n, 1, reinterpret_cast<const double2*>(s_n), nullptr, out, out);
  }

  // adjoint state [Y_n, Y_{n+1}] (eq. IMEX_adjoint), kept in the Y ring during the call
  spadj_status step_adjoint(Problem* p, int n, const double* x_n, const double* y_np1, const double* src, double* y_n,
                            double* gp_accum) override {
    if (n < 0) return p->fail(SPADJ_ERR_INVALID, "step: n < 0");
    if (gp_accum && !closure) return p->fail(SPADJ_ERR_INVALID, "step_adjoint: gp_accum but the problem has no parameters");
    const size_t sb = sbytes();
    const long long S = state_size;
    const double2* yin = reinterpret_cast<const double2*>(y_np1);
    double2* yout = reinterpret_cast<double2*>(y_n);
    // the seed map for index n: src (if any) as seed 0
    std::vector<int> sm(n + 1, -1);
    if (src) sm[n] = 0;
    SPADJ_CUDA_TRY(p, seedmap.ensure(sizeof(int) * (n + 1)));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(seedmap.ptr, sm.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, p->stream));
    if (closure && gp_accum) SPADJ_CUDA_TRY(p, cudaMemsetAsync(gp.ptr, 0, sizeof(double) * cnn::n_params(), p->stream));
    spadj_status st;
    if (!yin) {  // the seed step: no later adjoint variables, no vector-Jacobian product
      for (int i = 0; i < 2; ++i) SPADJ_CUDA_TRY(p, cudaMemsetAsync(Yr[i].ptr, 0, sb, p->stream));
      st = run_adjoint_seg(p, n, n, n, reinterpret_cast<const double2*>(x_n), seedmap.as<int>(),
                           reinterpret_cast<const double2*>(src), n == 0 ? y_n : nullptr, n);
    } else {
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(Yr[(n + 1) & 1].ptr, yin, sb, cudaMemcpyDeviceToDevice, p->stream));
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(Yr[n & 1].ptr, yin + S, sb, cudaMemcpyDeviceToDevice, p->stream));
      st = run_adjoint_seg(p, 1 << 29, n, n, reinterpret_cast<const double2*>(x_n), seedmap.as<int>(),
                           reinterpret_cast<const double2*>(src), n == 0 ? y_n : nullptr, 1 << 29);
    }
    if (st != SPADJ_OK) return st;
    if (n >= 1) SPADJ_CUDA_TRY(p, cudaMemcpyAsync(yout, Yr[n & 1].ptr, sb, cudaMemcpyDeviceToDevice, p->stream));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(yout + S, yin ? Yr[(n + 1) & 1].ptr : Yr[(n + 1) & 1].ptr, sb,
                                      cudaMemcpyDeviceToDevice, p->stream));
    if (closure && gp_accum) {
      add_kernel<<<64, 256, 0, p->stream>>>(gp_accum, gp.as<double>(), cnn::n_params());
      if ((st = check_launch(p, "gp accumulate")) != SPADJ_OK) return st;
    }
    return cudaStreamSynchronize(p->stream) == cudaSuccess ? SPADJ_OK : p->fail(SPADJ_ERR_CUDA, "sync");
  }

  // ---- learned closure ---------------------------------------------------------------------
  int cnn_grid(long long n) const { return (int)std::min<long long>((n + 255) / 256, 4096); }
  // thin-layer kernels: (pixel-channel tiles of 256 over one member's M^2 x C, members)
  dim3 thin_grid(int M, int C) const { return dim3((unsigned)(((long long)M * M * C + 255) / 256), (unsigned)nmem); }
  // one thread per pixel: (pixel tiles of 128, members)
  dim3 pixel_grid(int M) const { return dim3((unsigned)(((long long)M * M + 127) / 128), (unsigned)nmem); }
  int mma_grid(long long npix) const { return (int)std::min<long long>((npix + 63) / 64, 8192); }

  // One 32 -> 32 convolution of layer l (1 or 2) over all members: mode 0 forward hidden layer
  // (h, dact), 1 input gradient (fout), 2 pre-activation (fout, tests).  On the fifth-generation tensor
  // cores (tcgen05, accumulator in tensor memory; default) or, with spadj_set_option 11 = 0, the
  // warp-level mma.sync kernel (modes 0 and 1).
  int sm_count = 0;
  int tc_conv = 1;
  int thin_wgrad = 1;  // thin layers' weight gradients: 1 windowed (all taps per CTA), 0 one CTA per tap triple
  int thin_out = 1;    // thin layers' single-channel outputs: 1 windowed (32-channel side), 0 one thread per pixel
  bool halo_fits = true;                           // the halo-staged network kernels fit this grid
  static constexpr size_t kHaloSmemMax = 226 * 1024;  // opt-in shared memory per CTA less the static part
  DevBuf cnnerr;
  spadj_status conv32(Problem* p, int l, int mode, const __nv_bfloat16* in, __nv_bfloat16* h, float* da, float* fout) {
    const int M = hm[0].M, nb = nmem;
    const long long P = (long long)M * M * nb;
    if (tc_conv == 1 && halo_fits) {  // operand staged once per tile (halo), nine shifted descriptors
      const long long tiles = (long long)((M * (M + 2) + cnn::kTcRows - 1) / cnn::kTcRows) * nb;
      const int grid = (int)std::min<long long>(tiles, 3LL * sm_count);
      cnn::conv32_halo_kernel<<<grid, 128, cnn::halo_smem(M), p->stream>>>(
          l, M, nb, mode, in, wq.as<__nv_bfloat16>(), bq.as<float>(), h, da, fout, cnnerr.as<int>());
    } else if (tc_conv != 0) {  // operand gathered per tap
      const long long tiles = (P + cnn::kTcRows - 1) / cnn::kTcRows;
      const int grid = (int)std::min<long long>(tiles, 2LL * sm_count);
      cnn::conv32_tc_kernel<<<grid, 128, cnn::kTcSmem, p->stream>>>(l, M, nb, mode, in, wq.as<__nv_bfloat16>(),
                                                                     bq.as<float>(), h, da, fout, cnnerr.as<int>());
    } else {
      if (mode == 2) return p->fail(SPADJ_ERR_UNSUPPORTED, "closure conv: pre-activation output needs the tcgen05 kernel");
      cnn::conv32_mma_kernel<<<mma_grid(P), 128, 0, p->stream>>>(l, M, nb, mode, in, wq.as<__nv_bfloat16>(),
                                                                  bq.as<float>(), h, da, fout);
    }
    return check_launch(p, "closure conv");
  }

  spadj_status closure_conv_layer(Problem* p, int l, int mode, const void* in, float* out) {
    if (!closure) return p->fail(SPADJ_ERR_UNSUPPORTED, "closure_conv: the problem has no learned closure");
    if ((l != 1 && l != 2) || mode < 0 || mode > 2)
      return p->fail(SPADJ_ERR_INVALID, "closure_conv: layer must be 1 or 2 and mode 0, 1 or 2");
    const __nv_bfloat16* x = reinterpret_cast<const __nv_bfloat16*>(in);
    if (mode == 2)  // the forward epilogue: h into the layer's own activation buffer, 1 - tanh^2 into out
      return conv32(p, l, 0, x, hbuf[l].as<__nv_bfloat16>(), out, nullptr);
    return conv32(p, l, mode == 0 ? 2 : 1, x, nullptr, nullptr, out);
  }

  spadj_status check_cnn(Problem* p) {  // synchronises the stream
    int e = 0;
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(&e, cnnerr.ptr, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    if (e) {
      SPADJ_CUDA_TRY(p, cudaMemsetAsync(cnnerr.ptr, 0, sizeof(int), p->stream));
      return p->fail(SPADJ_ERR_TIMEOUT, "closure: a tensor-core convolution gave up waiting for its MMAs");
    }
    return SPADJ_OK;
  }

  spadj_status closure_forward(Problem* p, const KolArgs& A) {
    const int M = hm[0].M, nb = nmem;
    const long long P = (long long)M * M * nb;
    cudaEvent_t t = p->tic();
    cnn::quantize_kernel<<<cnn_grid(P), 256, 0, p->stream>>>(gridW.as<double>(), xq.as<__nv_bfloat16>(), (int)P);
    const __nv_bfloat16* in = xq.as<__nv_bfloat16>();
    for (int l = 0; l < cnn::kLayers; ++l) {
      const int co = (l == cnn::kLayers - 1) ? 1 : cnn::kHid;
      if (l == 1 || l == 2)  // 32 -> 32: tensor cores
        conv32(p, l, 0, in, hbuf[l].as<__nv_bfloat16>(), nullptr, nullptr);
      else if (l == 0)
        cnn::fwd0_kernel<<<pixel_grid(M), 128, 0, p->stream>>>(M, in, wq.as<__nv_bfloat16>(), bq.as<float>(),
                                                                hbuf[l].as<__nv_bfloat16>(), nullptr);
      else if (thin_out)
        cnn::thin_out_win_kernel<false><<<dim3(cnn::kThinBands, nb), 256, 0, p->stream>>>(
            M, in, wq.as<__nv_bfloat16>(), bq.as<float>(), corr.as<double>());
      else
        cnn::fwd_kernel<cnn::kHid, 1><<<thin_grid(M, co), 256, 0, p->stream>>>(
            l, M, in, wq.as<__nv_bfloat16>(), bq.as<float>(), nullptr, nullptr, corr.as<double>());
      if (l < 3) in = hbuf[l].as<__nv_bfloat16>();
    }
    closure_rows_kernel<<<dim3(M, nb), kKolThreads, smem, p->stream>>>(A, corr.as<double>(), 0);
    p->toc(t, KC_CNN, 2.0 * P * (9.0 * 32 + 2 * 9.0 * 32 * 32 + 9.0 * 32));
    return check_launch(p, "closure forward");
  }

  spadj_status closure_backward(Problem* p, const KolArgs& A) {
    const int M = hm[0].M, nb = nmem, np = cnn::n_params();
    const long long P = (long long)M * M * nb;
    cudaEvent_t t = p->tic();
    cnn::quantize_kernel<<<cnn_grid(P), 256, 0, p->stream>>>(gridW.as<double>(), xq.as<__nv_bfloat16>(), (int)P);
    const __nv_bfloat16* ins[4] = {xq.as<__nv_bfloat16>(), hbuf[0].as<__nv_bfloat16>(), hbuf[1].as<__nv_bfloat16>(),
                                   hbuf[2].as<__nv_bfloat16>()};
    for (int l = 0; l < 3; ++l) {
      if (l == 0)
        cnn::fwd0_kernel<<<pixel_grid(M), 128, 0, p->stream>>>(M, ins[l], wq.as<__nv_bfloat16>(), bq.as<float>(),
                                                                hbuf[l].as<__nv_bfloat16>(), dact[l].as<float>());
      else
        conv32(p, l, 0, ins[l], hbuf[l].as<__nv_bfloat16>(), dact[l].as<float>(), nullptr);
    }
    // The tensor-core convolutions and the layer-3 input gradient write the next layer's BF16
    // cotangent dz = bf16(din * dact) from their epilogue (two dz buffers in turn); the mma.sync form
    // writes din in FP32 and a separate pass forms dz.
    const bool fuse = tc_conv != 0;
    __nv_bfloat16* dzb[2] = {dz.as<__nv_bfloat16>(), dz2.as<__nv_bfloat16>()};
    int cur = 0;
    for (int l = cnn::kLayers - 1; l >= 0; --l) {
      const int co = (l == cnn::kLayers - 1) ? 1 : cnn::kHid, ci = (l == 0) ? 1 : cnn::kHid;
      __nv_bfloat16* dzc = dzb[cur];
      if (l == cnn::kLayers - 1)
        cnn::dz_kernel<<<cnn_grid(P), 256, 0, p->stream>>>(P, nullptr, nullptr, gridG.as<double>(), dzc);
      else if (!fuse)
        cnn::dz_kernel<<<cnn_grid(P * co), 256, 0, p->stream>>>(P * co, dh.as<float>(), dact[l].as<float>(), nullptr,
                                                                 dzc);
      if (l == 1 || l == 2) {  // 32 -> 32: tensor cores
        // the halo kernel also sums the bias gradient from its staged dz rows
        float* bpart = chunkbuf.as<float>() + (size_t)nb * 9 * kWgradChunks * 1024;
        const bool halo = tc_conv == 1 && halo_fits;
        if (halo)  // halo-staged operands, ldmatrix fragments, one warp per tap
          cnn::wgrad32_halo_kernel<<<dim3(kWgradChunks, nb), 288, cnn::wgrad_halo_smem(M), p->stream>>>(
              M, ins[l], dzc, chunkbuf.as<float>(), kWgradChunks, bpart);
        else
          cnn::wgrad32_mma_kernel<<<dim3(kWgradChunks, 9, nb), 128, 0, p->stream>>>(
              l, M, ins[l], dzc, chunkbuf.as<float>(), kWgradChunks);
        cnn::wgrad32_finish_kernel<<<dim3(36, nb), 256, 0, p->stream>>>(l, chunkbuf.as<float>(), kWgradChunks,
                                                                        part.as<float>(), np, halo ? bpart : nullptr);
        if (!halo) cnn::bgrad32_kernel<<<dim3(32, nb), 256, 0, p->stream>>>(l, M, dzc, part.as<float>(), np);
        if (fuse)
          conv32(p, l, 3, dzc, dzb[cur ^ 1], dact[l - 1].as<float>(), nullptr);
        else
          conv32(p, l, 1, dzc, nullptr, nullptr, dh.as<float>());
      } else if (l == 0) {
        if (thin_wgrad)
          cnn::wgrad_win_kernel<1, cnn::kHid><<<dim3(cnn::kThinSplits, nb), 256, 0, p->stream>>>(
              M, ins[l], dzc, chunkbuf.as<float>());
        else
          cnn::wgrad_kernel<1, cnn::kHid><<<dim3(4, nb, cnn::kThinSplits), 256, 0, p->stream>>>(
              l, M, ins[l], dzc, chunkbuf.as<float>());
        cnn::wgrad_finish_kernel<<<nb, 320, 0, p->stream>>>(l, chunkbuf.as<float>(), part.as<float>(), np);
        if (thin_out)
          cnn::thin_out_win_kernel<true><<<dim3(cnn::kThinBands, nb), 256, 0, p->stream>>>(
              M, dzc, wq.as<__nv_bfloat16>(), bq.as<float>(), corr.as<double>());
        else
          cnn::dgrad_kernel<1, cnn::kHid><<<thin_grid(M, ci), 256, 0, p->stream>>>(
              l, M, dzc, wq.as<__nv_bfloat16>(), nullptr, corr.as<double>());
      } else {
        if (thin_wgrad)
          cnn::wgrad_win_kernel<cnn::kHid, 1><<<dim3(cnn::kThinSplits, nb), 256, 0, p->stream>>>(
              M, ins[l], dzc, chunkbuf.as<float>());
        else
          cnn::wgrad_kernel<cnn::kHid, 1><<<dim3(4, nb, cnn::kThinSplits), 256, 0, p->stream>>>(
              l, M, ins[l], dzc, chunkbuf.as<float>());
        cnn::wgrad_finish_kernel<<<nb, 320, 0, p->stream>>>(l, chunkbuf.as<float>(), part.as<float>(), np);
        cnn::dgrad3_kernel<<<pixel_grid(M), 128, 0, p->stream>>>(
            M, dzc, wq.as<__nv_bfloat16>(), fuse ? nullptr : dh.as<float>(), fuse ? dact[l - 1].as<float>() : nullptr,
            fuse ? dzb[cur ^ 1] : nullptr);
      }
      if (fuse) cur ^= 1;
    }
    cnn::reduce_params_kernel<<<64, 256, 0, p->stream>>>(part.as<float>(), nb, np, gp.as<double>());
    closure_rows_kernel<<<dim3(M, nb), kKolThreads, smem, p->stream>>>(A, corr.as<double>(), 1);
    p->toc(t, KC_CNN, 6.0 * P * (9.0 * 32 + 2 * 9.0 * 32 * 32 + 9.0 * 32));
    return check_launch(p, "closure backward");
  }

  // spectral truncation of fine members (n_fine modes) to this uniform-resolution batch
  spadj_status restrict_from(Problem* p, int n_fine, const double* fine, double* coarse) {
    const int Nc = hm[0].N;
    for (auto& m : hm)
      if (m.N != Nc) return p->fail(SPADJ_ERR_UNSUPPORTED, "restrict: the batch must have one resolution");
    if (n_fine < Nc || n_fine % 2 != 0) return p->fail(SPADJ_ERR_INVALID, "restrict: n_fine must be even and >= n[0]");
    const long long n = (long long)(Nc / 2) * Nc * nmem;
    const int grid = (int)std::min<long long>((n + 255) / 256, 4096);
    restrict_kernel<<<grid, 256, 0, p->stream>>>(reinterpret_cast<const double2*>(fine), n_fine, Nc, nmem,
                                                 reinterpret_cast<double2*>(coarse));
    return check_launch(p, "restrict");
  }

  spadj_status adam(Problem* p, const double* g, int t, double lr, double b1, double b2, double eps, double* m,
                    double* v, double* params) {
    if (!closure) return p->fail(SPADJ_ERR_UNSUPPORTED, "adam: the problem has no learned closure");
    if (t < 1 || !(lr > 0) || !(b1 >= 0 && b1 < 1) || !(b2 >= 0 && b2 < 1) || !(eps > 0))
      return p->fail(SPADJ_ERR_INVALID, "adam: need t >= 1, lr > 0, 0 <= b1, b2 < 1, eps > 0");
    const int n = cnn::n_params();
    const double c1 = 1.0 - std::pow(b1, t), c2 = 1.0 - std::pow(b2, t);
    adam_kernel<<<(n + 255) / 256, 256, 0, p->stream>>>(n, g, b1, b2, lr, eps, c1, c2, m, v, params);
    return check_launch(p, "adam");
  }

  spadj_status set_params(Problem* p, const double* params) {
    if (!closure) return p->fail(SPADJ_ERR_UNSUPPORTED, "set_params: the problem has no learned closure");
    const size_t np = (size_t)cnn::n_params();
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(pbuf.ptr, params, sizeof(double) * np, cudaMemcpyDeviceToDevice, p->stream));
    cnn::convert_kernel<<<64, 256, 0, p->stream>>>(pbuf.as<double>(), wq.as<__nv_bfloat16>(), bq.as<float>());
    return check_launch(p, "closure convert");
  }

  spadj_status transform(Problem* p, int, const double*, double*) override {
    return p->fail(SPADJ_ERR_UNSUPPORTED, "kolmogorov: standalone transforms are not exposed");
  }

  spadj_status eval_F(Problem* p, int mode, const double* x, const double*, double* out) override {
    if (mode != 0) return p->fail(SPADJ_ERR_UNSUPPORTED, "kolmogorov: JVP/VJP of F are exercised through spadj_vjp");
    KolArgs A = base_args();
    A.adjoint = 0;
    A.fonly = 1;
    A.nstage = 2;
    A.S = 1;
    A.x0 = reinterpret_cast<const double2*>(x);
    A.out = reinterpret_cast<double2*>(out);
    const int keep = persistent;
    persistent = 0;
    spadj_status s = launch(p, A);
    persistent = keep;
    return s;
  }

  spadj_status forward(Problem* p, int n_steps, const double* x0, double* x_out, double* traj) override {
    if (n_steps < 1) return p->fail(SPADJ_ERR_INVALID, "forward: n_steps < 1");
    return run_forward(p, n_steps, x0, x_out, reinterpret_cast<double2*>(traj));
  }

  spadj_status tangent(Problem* p, int, const double*, const double*, double*) override {
    return p->fail(SPADJ_ERR_UNSUPPORTED, "kolmogorov: tangent sweep not provided");
  }

  spadj_status ensure_traj(Problem* p, int n_steps) {
    SPADJ_CUDA_TRY(p, trajbuf.ensure(sizeof(double2) * (size_t)state_size * (size_t)(n_steps + 1)));
    return SPADJ_OK;
  }

  spadj_status adjoint(Problem* p, int n_steps, const double* traj, const double* y_final, double* grad,
                       double* grad_p) override {
    if (n_steps < 1) return p->fail(SPADJ_ERR_INVALID, "adjoint: n_steps < 1");
    if (grad_p && !closure) return p->fail(SPADJ_ERR_INVALID, "adjoint: grad_p requested but the problem has no parameters");
    std::vector<int> seed_at(n_steps + 1, -1);
    seed_at[n_steps] = 0;
    if (closure) SPADJ_CUDA_TRY(p, cudaMemsetAsync(gp.ptr, 0, sizeof(double) * cnn::n_params(), p->stream));
    spadj_status s = run_adjoint(p, n_steps, const_cast<double2*>(reinterpret_cast<const double2*>(traj)), seed_at,
                                 reinterpret_cast<const double2*>(y_final), grad);
    if (s != SPADJ_OK) return s;
    if (grad_p)
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(grad_p, gp.ptr, sizeof(double) * cnn::n_params(), cudaMemcpyDeviceToDevice,
                                        p->stream));
    return SPADJ_OK;
  }

  // checkpointed sweeps: ckpt_slots in 1..n_steps-1 segments with device-resident starts, or the
  // host slots of spadj_set_option 9 (page-locked segment starts)
  bool segmented(Problem* p, int n_steps, int ckpt_slots) const {
    return p->host_slots > 0 || (ckpt_slots > 0 && ckpt_slots < n_steps);
  }

  spadj_status vjp(Problem* p, const double* x0, int n_steps, int ckpt_slots, const std::vector<int>& seed_at,
                   const double* seeds, double* grad) override {
    if (n_steps < 1) return p->fail(SPADJ_ERR_INVALID, "vjp: n_steps < 1");
    if (segmented(p, n_steps, ckpt_slots)) {
      if (closure) SPADJ_CUDA_TRY(p, cudaMemsetAsync(gp.ptr, 0, sizeof(double) * cnn::n_params(), p->stream));
      const bool host = p->host_slots > 0;
      return reverse_seg(p, x0, n_steps, host ? p->host_slots : ckpt_slots, host, false, seed_at,
                         reinterpret_cast<const double2*>(seeds), grad, nullptr);
    }
    spadj_status s = ensure_traj(p, n_steps);
    if (s != SPADJ_OK) return s;
    if ((s = run_forward(p, n_steps, x0, tmp.as<double>(), trajbuf.as<double2>())) != SPADJ_OK) return s;
    return run_adjoint(p, n_steps, trajbuf.as<double2>(), seed_at, reinterpret_cast<const double2*>(seeds), grad);
  }

  spadj_status set_observations(Problem* p, int n, const int* steps, const double* obs, int kmax) {
    if (n < 1 || !steps || !obs || kmax < 0) return p->fail(SPADJ_ERR_INVALID, "set_observations: bad arguments");
    for (int i = 0; i < n; ++i)
      if (steps[i] < 1 || (i > 0 && steps[i] <= steps[i - 1]))
        return p->fail(SPADJ_ERR_INVALID, "set_observations: steps must be increasing and >= 1");
    n_obs = n;
    obs_kmax = kmax;
    obs_steps_h.assign(steps, steps + n);
    SPADJ_CUDA_TRY(p, obsbuf.ensure(sizeof(double2) * (size_t)state_size * n));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(obsbuf.ptr, obs, sizeof(double2) * (size_t)state_size * n, cudaMemcpyDeviceToDevice,
                                      p->stream));
    SPADJ_CUDA_TRY(p, obsteps.ensure(sizeof(int) * n));
    SPADJ_CUDA_TRY(p, cudaMemcpyAsync(obsteps.ptr, steps, sizeof(int) * n, cudaMemcpyHostToDevice, p->stream));
    SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    return SPADJ_OK;
  }

  spadj_status objective(Problem* p, int, const double*, const double*, double*, double*) override {
    return p->fail(SPADJ_ERR_UNSUPPORTED, "kolmogorov: the 4D-Var objective is evaluated inside spadj_gradient");
  }

  spadj_status gradient(Problem* p, const double* x0, int n_steps, int objective_kind, const double*, int ckpt_slots,
                        double* J_host, double* grad, double* grad_p) override {
    if (objective_kind != SPADJ_OBJ_FOURDVAR) return p->fail(SPADJ_ERR_UNSUPPORTED, "kolmogorov: objective must be FOURDVAR");
    if (n_obs < 1) return p->fail(SPADJ_ERR_INVALID, "kolmogorov: call spadj_set_observations first");
    if (obs_steps_h.back() > n_steps) return p->fail(SPADJ_ERR_INVALID, "kolmogorov: observation step beyond n_steps");
    if (grad_p && !closure) return p->fail(SPADJ_ERR_INVALID, "gradient: grad_p requested but the problem has no parameters");
    if (segmented(p, n_steps, ckpt_slots)) {
      if (closure) SPADJ_CUDA_TRY(p, cudaMemsetAsync(gp.ptr, 0, sizeof(double) * cnn::n_params(), p->stream));
      const bool host = p->host_slots > 0;
      std::vector<double> Jl(nmem, 0.0);
      spadj_status s = reverse_seg(p, x0, n_steps, host ? p->host_slots : ckpt_slots, host, true, {}, nullptr, grad,
                                   Jl.data());
      if (s != SPADJ_OK) return s;
      if (grad_p)
        SPADJ_CUDA_TRY(p, cudaMemcpyAsync(grad_p, gp.ptr, sizeof(double) * cnn::n_params(), cudaMemcpyDeviceToDevice,
                                          p->stream));
      if (closure && J_host && (s = check_cnn(p)) != SPADJ_OK) return s;
      if (J_host) {
        for (int b = 0; b < nmem; ++b) {
          J_host[b] = Jl[b];
          if (!std::isfinite(J_host[b])) return p->fail(SPADJ_ERR_NONFINITE, "kolmogorov: objective is not finite");
        }
      }
      return SPADJ_OK;
    }
    spadj_status s = ensure_traj(p, n_steps);
    if (s != SPADJ_OK) return s;
    if ((s = run_forward(p, n_steps, x0, tmp.as<double>(), trajbuf.as<double2>())) != SPADJ_OK) return s;
    SPADJ_CUDA_TRY(p, seedbuf.ensure(sizeof(double2) * (size_t)state_size * n_obs));
    SPADJ_CUDA_TRY(p, partial.ensure(sizeof(double) * (size_t)nmem * n_obs));
    SPADJ_CUDA_TRY(p, Jd.ensure(sizeof(double) * nmem));
    cudaEvent_t t = p->tic();
    fourdvar_kernel<<<dim3(nmem, n_obs), kKolThreads, 0, p->stream>>>(dmem.as<KMember>(), trajbuf.as<double2>(),
                                                                      obsteps.as<int>(), obsbuf.as<double2>(), state_size,
                                                                      obs_kmax, seedbuf.as<double2>(),
                                                                      partial.as<double>(), n_obs);
    sum_rows_kernel<<<(nmem + 127) / 128, 128, 0, p->stream>>>(partial.as<double>(), n_obs, nmem, Jd.as<double>());
    p->toc(t, KC_OBJECTIVE, 4.0 * state_size * n_obs);
    if ((s = check_launch(p, "kolmogorov 4dvar")) != SPADJ_OK) return s;
    std::vector<int> seed_at(n_steps + 1, -1);
    for (int i = 0; i < n_obs; ++i) seed_at[obs_steps_h[i]] = i;
    if (closure) SPADJ_CUDA_TRY(p, cudaMemsetAsync(gp.ptr, 0, sizeof(double) * cnn::n_params(), p->stream));
    if ((s = run_adjoint(p, n_steps, trajbuf.as<double2>(), seed_at, seedbuf.as<double2>(), grad)) != SPADJ_OK) return s;
    if (grad_p) {
      if (!closure) return p->fail(SPADJ_ERR_INVALID, "gradient: grad_p requested but the problem has no parameters");
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(grad_p, gp.ptr, sizeof(double) * cnn::n_params(), cudaMemcpyDeviceToDevice,
                                        p->stream));
    }
    if (closure && J_host) {
      spadj_status e = check_cnn(p);
      if (e != SPADJ_OK) return e;
    }
    if (J_host) {
      SPADJ_CUDA_TRY(p, cudaMemcpyAsync(J_host, Jd.ptr, sizeof(double) * nmem, cudaMemcpyDeviceToHost, p->stream));
      SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
      for (int b = 0; b < nmem; ++b)
        if (!std::isfinite(J_host[b])) return p->fail(SPADJ_ERR_NONFINITE, "kolmogorov: objective is not finite");
    }
    return SPADJ_OK;
  }

  spadj_status set_option(Problem* p, int option, int value) {
    switch (option) {
      case 0:
        persistent = value ? 1 : 0;
        return SPADJ_OK;
      case 1:
        if (value < 1 || value > 64) return p->fail(SPADJ_ERR_INVALID, "set_option: column tile must be 1..64");
        CW = value; grid_persistent = 0; return sync_members(p);
      case 2:
        if (value < 1 || value > 64) return p->fail(SPADJ_ERR_INVALID, "set_option: row tile must be 1..64");
        RW = value; grid_persistent = 0; return sync_members(p);
      case 3:
        if (value < 0 || value > 32) return p->fail(SPADJ_ERR_INVALID, "set_option: CTAs per SM must be 0..32");
        ctas_per_sm = value; grid_persistent = 0; return SPADJ_OK;
      case 4:  // bounded-wait iteration limit (0 = default)
        spin_limit = value > 0 ? (unsigned)value : kSpinLimit; return SPADJ_OK;
      case 5:  // failure-path test: member whose completion is never signalled (-1 = off)
        if (value < -1 || value >= nmem) return p->fail(SPADJ_ERR_INVALID, "set_option: member out of range");
        drop_signal_member = value; return SPADJ_OK;
      case 11:  // closure convolutions: tcgen05 with a halo-staged operand (1), tcgen05 with the operand
                // gathered per tap (2), or mma.sync (0)
        if (value < 0 || value > 2) return p->fail(SPADJ_ERR_INVALID, "set_option 11: 0, 1 or 2");
        tc_conv = value; return SPADJ_OK;
      case 13:  // thin layers' weight gradients: windowed (1) or one CTA per tap triple (0)
        if (value < 0 || value > 1) return p->fail(SPADJ_ERR_INVALID, "set_option 13: 0 or 1");
        thin_wgrad = value; return SPADJ_OK;
      case 14:  // thin layers' single-channel outputs: windowed (1) or one thread per pixel (0)
        if (value < 0 || value > 1) return p->fail(SPADJ_ERR_INVALID, "set_option 14: 0 or 1");
        thin_out = value; return SPADJ_OK;
      default: return p->fail(SPADJ_ERR_INVALID, "set_option: unknown option");
    }
  }

  // Time a short forward sweep for each candidate tiling and keep the fastest; results are
  // cached per process by the batch's resolutions.
  spadj_status autotune(Problem* p) {
    static std::map<std::vector<int>, std::vector<int>> cache;
    std::vector<int> key;
    for (auto& m : hm) key.push_back(m.N);
    auto it = cache.find(key);
    if (it != cache.end()) {
      CW = it->second[0]; RW = it->second[1]; ctas_per_sm = it->second[2]; grid_persistent = 0;
      return sync_members(p);
    }
    spadj_status s;
    // probe input: zero state is valid (forcing drives it)
    SPADJ_CUDA_TRY(p, cudaMemsetAsync(Yr[0].ptr, 0, sizeof(double2) * state_size, p->stream));
    double best = 1e300;
    std::vector<int> bestv = {CW, RW, ctas_per_sm};
    const int keep_p = persistent;
    persistent = 1;
    for (int cw : {2, 4, 8})
      for (int rw : {1, 2, 4})
        for (int cps : {0, 2}) {
          CW = cw; RW = rw; ctas_per_sm = cps; grid_persistent = 0;
          if ((s = sync_members(p)) != SPADJ_OK) return s;
          SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
          auto t0 = std::chrono::steady_clock::now();
          if ((s = run_forward(p, 4, Yr[0].as<double>(), Yr[1].as<double>(), nullptr)) != SPADJ_OK) return s;
          SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
          const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
          if (el < best) { best = el; bestv = {cw, rw, cps}; }
        }
    persistent = keep_p;
    cache[key] = bestv;
    CW = bestv[0]; RW = bestv[1]; ctas_per_sm = bestv[2]; grid_persistent = 0;
    return sync_members(p);
  }

  ~Kol() override {
    for (DevBuf* b : {&gridW, &gridG, &corr, &xq, &hbuf[0], &hbuf[1], &hbuf[2], &dact[0], &dact[1], &dact[2], &dh, &dz, &dz2,
                      &pbuf, &wq, &bq, &part, &gp, &chunkbuf})
      b->release();
    for (DevBuf* b : {&dmem, &tables, &Xr[0], &Xr[1], &Fr[0], &Fr[1], &Yr[0], &Yr[1], &mixA, &mixB, &ctr, &trajbuf,
                      &seedbuf, &seedmap, &obsbuf, &obsteps, &partial, &Jd, &tmp, &segx0, &segbuf, &rsbuf, &cslots,
                      &obsstates, &obsidx, &cnnerr})
      b->release();
    hcslots.release();
  }
};

}  // namespace

EqImpl* make_kolmogorov(Problem* p, spadj_status* st) {
  Kol* k = new Kol();
  *st = k->init(p);
  if (*st != SPADJ_OK) {
    delete k;
    return nullptr;
  }
  return k;
}

spadj_status kol_set_observations(EqImpl* impl, Problem* p, int n, const int* steps, const double* obs, int kmax) {
  Kol* k = dynamic_cast<Kol*>(impl);
  if (!k) return p->fail(SPADJ_ERR_UNSUPPORTED, "set_observations: only defined for the Kolmogorov batch");
  return k->set_observations(p, n, steps, obs, kmax);
}

spadj_status kol_set_option(EqImpl* impl, Problem* p, int option, int value) {
  Kol* k = dynamic_cast<Kol*>(impl);
  if (!k) return p->fail(SPADJ_ERR_UNSUPPORTED, "set_option: only defined for the Kolmogorov batch");
  return k->set_option(p, option, value);
}

spadj_status kol_set_params(EqImpl* impl, Problem* p, const double* params) {
  Kol* k = dynamic_cast<Kol*>(impl);
  if (!k) return p->fail(SPADJ_ERR_UNSUPPORTED, "set_params: only defined for the Kolmogorov batch with a closure");
  return k->set_params(p, params);
}

spadj_status kol_restrict(EqImpl* impl, Problem* p, int n_fine, const double* fine, double* coarse) {
  Kol* k = dynamic_cast<Kol*>(impl);
  if (!k) return p->fail(SPADJ_ERR_UNSUPPORTED, "restrict: only defined for SPADJ_KOLMOGOROV2D");
  return k->restrict_from(p, n_fine, fine, coarse);
}

spadj_status kol_adam(EqImpl* impl, Problem* p, const double* g, int t, double lr, double b1, double b2, double eps,
                      double* m, double* v, double* params) {
  Kol* k = dynamic_cast<Kol*>(impl);
  if (!k) return p->fail(SPADJ_ERR_UNSUPPORTED, "adam: only defined for SPADJ_KOLMOGOROV2D with a closure");
  return k->adam(p, g, t, lr, b1, b2, eps, m, v, params);
}

spadj_status kol_closure_conv(EqImpl* impl, Problem* p, int layer, int mode, const void* in, float* out) {
  Kol* k = dynamic_cast<Kol*>(impl);
  if (!k) return p->fail(SPADJ_ERR_UNSUPPORTED, "closure_conv: only defined for SPADJ_KOLMOGOROV2D with a closure");
  spadj_status s = k->closure_conv_layer(p, layer, mode, in, out);
  if (s != SPADJ_OK) return s;
  return k->check_cnn(p);
}

spadj_status kol_autotune(EqImpl* impl, Problem* p) {
  Kol* k = dynamic_cast<Kol*>(impl);
  if (!k) return p->fail(SPADJ_ERR_UNSUPPORTED, "autotune: only defined for the Kolmogorov batch");
  return k->autotune(p);
}

}  // namespace spadj
