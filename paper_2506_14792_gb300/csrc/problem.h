// Internal problem object behind the opaque spadj_problem handle.
#pragma once
#include <cuda_runtime.h>

#include <cstdio>
#include <string>
#include <vector>

#include "pdl.cuh"
#include "spadj.h"

namespace spadj {

// Return an error status with a message recorded on the problem.
#define SPADJ_CUDA_TRY(prob, expr)                                                        \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      (prob)->set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));             \
      return e_ == cudaErrorMemoryAllocation ? SPADJ_ERR_NOMEM : SPADJ_ERR_CUDA;         \
    }                                                                                    \
  } while (0)

// Device buffer owned by the library (grown on demand, freed with the problem).
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t nbytes) {
    if (nbytes <= bytes) return cudaSuccess;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&ptr, nbytes);
    if (e == cudaSuccess) bytes = nbytes;
    return e;
  }
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
  }
  template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// Page-locked host buffer owned by the library (grown on demand, freed with the problem);
// the host tier of the two-level checkpoint schedule.
struct HostBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t nbytes) {
    if (nbytes <= bytes) return cudaSuccess;
    if (ptr) cudaFreeHost(ptr);
    ptr = nullptr;
    bytes = 0;
    cudaError_t e = cudaHostAlloc(&ptr, nbytes, cudaHostAllocDefault);
    if (e == cudaSuccess) bytes = nbytes;
    return e;
  }
  void release() {
    if (ptr) cudaFreeHost(ptr);
    ptr = nullptr;
    bytes = 0;
  }
  template <class T> T* as() const { return static_cast<T*>(ptr); }
};

struct Problem;

// One equation set's implementation.  Every method runs asynchronously on prob->stream
// unless it writes host memory.
struct EqImpl {
  virtual ~EqImpl() {}
  virtual size_t state_len(int which) const = 0;
  virtual spadj_status transform(Problem* p, int kind, const double* in, double* out) = 0;
  virtual spadj_status eval_F(Problem* p, int mode, const double* x, const double* dx, double* out) = 0;
  virtual spadj_status forward(Problem* p, int n_steps, const double* x0, double* x_out, double* traj) = 0;
  virtual spadj_status tangent(Problem* p, int n_steps, const double* x0, const double* dx0, double* dx_out) = 0;
  virtual spadj_status adjoint(Problem* p, int n_steps, const double* traj, const double* y_final,
                               double* grad_x0, double* grad_p) = 0;
  virtual spadj_status objective(Problem* p, int objective, const double* obj_data, const double* x,
                                 double* J_dev, double* seed) = 0;
  virtual spadj_status gradient(Problem* p, const double* x0, int n_steps, int objective,
                                const double* obj_data, int ckpt_slots, double* J_host, double* grad_x0,
                                double* grad_p) = 0;
  // Reverse sweep seeded by caller cotangents: seed_at[n] indexes `seeds` for X_n (or -1).
  virtual spadj_status vjp(Problem* p, const double* x0, int n_steps, int ckpt_slots,
                           const std::vector<int>& seed_at, const double* seeds, double* grad_x0) = 0;
  // One step at a time (spadj_step_forward / _tangent / _adjoint).  step_blocks(0): state vectors
  // in the restart state of one step, step_blocks(1): in the adjoint state; 0 = not provided.
  virtual int step_blocks(int which) const { (void)which; return 0; }
  virtual spadj_status step_forward(Problem* p, int n, const double* s_n, double* s_np1) {
    (void)n; (void)s_n; (void)s_np1;
    return step_unsupported(p);
  }
  virtual spadj_status step_tangent(Problem* p, int n, const double* s_n, const double* ds_n, double* ds_np1) {
    (void)n; (void)s_n; (void)ds_n; (void)ds_np1;
    return step_unsupported(p);
  }
  virtual spadj_status step_adjoint(Problem* p, int n, const double* x_n, const double* y_np1, const double* src,
                                    double* y_n, double* gp_accum) {
    (void)n; (void)x_n; (void)y_np1; (void)src; (void)y_n; (void)gp_accum;
    return step_unsupported(p);
  }
  static spadj_status step_unsupported(Problem* p);
};

// Optional per-kernel-class timing: CUDA events recorded on the problem's stream around
// every launch of the library, with the algorithmic FP64 flop count of that launch.
enum KernelClass { KC_ZTRANSFORM = 0, KC_XFFT = 1, KC_POINTWISE = 2, KC_SOLVE = 3, KC_OBJECTIVE = 4, KC_FUSED = 5,
                   KC_YFFT = 6, KC_GRAM = 7, KC_CNN = 8, KC_COUNT = 9 };

struct Timing {
  bool enabled = false;
  struct Rec { int kc; cudaEvent_t a, b; double flops; };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  double ms[KC_COUNT] = {0}, flops[KC_COUNT] = {0};
  long launches[KC_COUNT] = {0};
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  void reset() {
    collect();
    for (int i = 0; i < KC_COUNT; ++i) { ms[i] = 0; flops[i] = 0; launches[i] = 0; }
  }
  void collect() {
    for (Rec& r : pending) {
      cudaEventSynchronize(r.b);
      float t = 0.f;
      cudaEventElapsedTime(&t, r.a, r.b);
      ms[r.kc] += t;
      flops[r.kc] += r.flops;
      launches[r.kc] += 1;
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    pending.clear();
  }
  ~Timing() {
    collect();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

struct Problem {
  spadj_desc desc{};
  cudaStream_t stream = nullptr;
  std::string err;
  EqImpl* impl = nullptr;
  Timing timing;
  bool pdl = false;          // programmatic dependent launch of consecutive kernels (spadj_set_option 6)
  bool fuse_columns = true;  // RB: fused fold + solve + expand cluster kernel (spadj_set_option 7)
  int x_rows = 0;            // x-FFT rows per CTA: 0 = tuned at creation, else 1, 2 or 4 (option 8)
  int host_slots = 0;        // host checkpoint slots of the two-level schedule, 0 = device only (option 9)
  bool bulk_staging = true;  // RB fused column stages: operator block by one bulk copy (option 10)
  int cou_band = -1;         // Couette step solves: banded (1), dense Phi (0), by size (-1) (option 12)
  cudaEvent_t tic() {
    if (!timing.enabled) return nullptr;
    cudaEvent_t e = timing.get();
    cudaEventRecord(e, stream);
    return e;
  }
  void toc(cudaEvent_t a, int kc, double flops) {
    if (!a) return;
    cudaEvent_t b = timing.get();
    cudaEventRecord(b, stream);
    timing.pending.push_back({kc, a, b, flops});
    if (timing.pending.size() > 4096) timing.collect();
  }
  void set_error(const std::string& s) { err = s; }
  spadj_status fail(spadj_status st, const std::string& s) {
    err = s;
    return st;
  }
};

inline spadj_status EqImpl::step_unsupported(Problem* p) {
  return p->fail(SPADJ_ERR_UNSUPPORTED, "step entry points are not provided for this equation set");
}

// Launch-error check after a kernel launch.
inline spadj_status check_launch(Problem* p, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return p->fail(SPADJ_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return SPADJ_OK;
}

// Factories (one per equation set).
EqImpl* make_burgers(Problem* p, spadj_status* st);
spadj_status burgers_set_dt_schedule(EqImpl* impl, Problem* p, int n, const double* dts);
EqImpl* make_rb(Problem* p, spadj_status* st);
spadj_status rb_pencil_solve(EqImpl* impl, Problem* p, int transpose, const double* v, double* x);
spadj_status rb_set_dt_schedule(EqImpl* impl, Problem* p, int n, const double* dts);
EqImpl* make_kolmogorov(Problem* p, spadj_status* st);
EqImpl* make_shear_evp(Problem* p, spadj_status* st);
spadj_status evp_eigen(EqImpl* impl, Problem* p, int n_pencils, const double* prm, const double* shift, int n_iter,
                       double* x, double* psi, double* out);
spadj_status kol_set_observations(EqImpl* impl, Problem* p, int n, const int* steps, const double* obs, int kmax);
spadj_status kol_set_option(EqImpl* impl, Problem* p, int option, int value);
spadj_status kol_autotune(EqImpl* impl, Problem* p);
spadj_status kol_set_params(EqImpl* impl, Problem* p, const double* params);
spadj_status kol_restrict(EqImpl* impl, Problem* p, int n_fine, const double* fine, double* coarse);
spadj_status kol_closure_conv(EqImpl* impl, Problem* p, int layer, int mode, const void* in, float* out);
spadj_status kol_adam(EqImpl* impl, Problem* p, const double* g, int t, double lr, double b1, double b2, double eps,
                      double* m, double* v, double* params);
spadj_status rb_transform_noalloc(EqImpl* impl, Problem* p, int kind, const double* in, double* out);
EqImpl* make_couette(Problem* p, spadj_status* st);
spadj_status cou_pencil_solve(EqImpl* impl, Problem* p, int transpose, const double* v, double* x);
spadj_status cou_resolvent(EqImpl* impl, Problem* p, double omega, int n_iter, double* f, double* gains);
spadj_status cou_hvp(EqImpl* impl, Problem* p, const double* x0, const double* v, int n_steps, double* hv);

}  // namespace spadj

struct spadj_problem : public spadj::Problem {};
