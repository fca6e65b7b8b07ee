// C-ABI entry points declared in include/spadj.h: argument checks and dispatch to the
// equation set's implementation.  No arithmetic of the method happens here.
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "couette_setup.h"
#include "problem.h"
#include "revolve.h"

using spadj::Problem;

namespace {
thread_local std::string g_create_error = "no error";

bool bad_ptr(const void* p) { return p == nullptr; }
}  // namespace

extern "C" {

spadj_status spadj_create(const spadj_desc* desc, void* cuda_stream, spadj_problem** out) {
  if (!desc || !out) {
    g_create_error = "spadj_create: desc and out must be non-NULL";
    return SPADJ_ERR_INVALID;
  }
  *out = nullptr;
  if (desc->batch < 1 || (desc->eq != SPADJ_SHEAR_EVP && !(desc->dt > 0.0))) {
    g_create_error = "spadj_create: batch must be >= 1 and dt > 0";
    return SPADJ_ERR_INVALID;
  }
  spadj_problem* p = new (std::nothrow) spadj_problem();
  if (!p) {
    g_create_error = "spadj_create: out of host memory";
    return SPADJ_ERR_NOMEM;
  }
  p->desc = *desc;
  p->stream = static_cast<cudaStream_t>(cuda_stream);
  spadj_status st = SPADJ_ERR_UNSUPPORTED;
  switch (desc->eq) {
    case SPADJ_BURGERS1D: p->impl = spadj::make_burgers(p, &st); break;
    case SPADJ_RB2D: p->impl = spadj::make_rb(p, &st); break;
    case SPADJ_KOLMOGOROV2D: p->impl = spadj::make_kolmogorov(p, &st); break;
    case SPADJ_COUETTE3D: p->impl = spadj::make_couette(p, &st); break;
    case SPADJ_SHEAR_EVP: p->impl = spadj::make_shear_evp(p, &st); break;
    default: p->err = "spadj_create: unknown equation set"; break;
  }
  if (st != SPADJ_OK || !p->impl) {
    g_create_error = p->err.empty() ? "spadj_create failed" : p->err;
    delete p->impl;
    delete p;
    return st == SPADJ_OK ? SPADJ_ERR_INVALID : st;
  }
  *out = p;
  return SPADJ_OK;
}

spadj_status spadj_destroy(spadj_problem* p) {
  if (!p) return SPADJ_ERR_INVALID;
  cudaStreamSynchronize(p->stream);
  delete p->impl;
  delete p;
  return SPADJ_OK;
}

size_t spadj_state_len(const spadj_problem* p, int which) {
  if (!p || !p->impl) return 0;
  if (which == 4 || which == 5) return (size_t)p->impl->step_blocks(which - 4) * p->impl->state_len(0);
  return p->impl->state_len(which);
}

spadj_status spadj_transform(spadj_problem* p, int kind, const double* in, double* out) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(in) || bad_ptr(out)) return p->fail(SPADJ_ERR_INVALID, "transform: NULL array");
  return p->impl->transform(p, kind, in, out);
}

spadj_status spadj_transform_noalloc(spadj_problem* p, int kind, const double* in, double* out) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(in) || bad_ptr(out)) return p->fail(SPADJ_ERR_INVALID, "transform_noalloc: NULL array");
  return spadj::rb_transform_noalloc(p->impl, p, kind, in, out);
}

spadj_status spadj_eval_F(spadj_problem* p, const double* x, double* f) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(x) || bad_ptr(f)) return p->fail(SPADJ_ERR_INVALID, "eval_F: NULL array");
  return p->impl->eval_F(p, 0, x, nullptr, f);
}

spadj_status spadj_eval_F_jvp(spadj_problem* p, const double* x, const double* dx, double* df) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(x) || bad_ptr(dx) || bad_ptr(df)) return p->fail(SPADJ_ERR_INVALID, "eval_F_jvp: NULL array");
  return p->impl->eval_F(p, 1, x, dx, df);
}

spadj_status spadj_eval_F_vjp(spadj_problem* p, const double* x, const double* y, double* out) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(x) || bad_ptr(y) || bad_ptr(out)) return p->fail(SPADJ_ERR_INVALID, "eval_F_vjp: NULL array");
  return p->impl->eval_F(p, 2, x, y, out);
}

spadj_status spadj_solve(spadj_problem* p, int transpose, const double* v, double* x) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(v) || bad_ptr(x)) return p->fail(SPADJ_ERR_INVALID, "solve: NULL array");
  if (p->desc.eq == SPADJ_COUETTE3D) return spadj::cou_pencil_solve(p->impl, p, transpose, v, x);
  return spadj::rb_pencil_solve(p->impl, p, transpose, v, x);
}

spadj_status spadj_hvp(spadj_problem* p, const double* x0, const double* v, int n_steps, double* hv) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(x0) || bad_ptr(v) || bad_ptr(hv)) return p->fail(SPADJ_ERR_INVALID, "hvp: NULL array");
  return spadj::cou_hvp(p->impl, p, x0, v, n_steps, hv);
}

spadj_status spadj_resolvent(spadj_problem* p, double omega, int n_iter, double* f, double* gains) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(f) || bad_ptr(gains)) return p->fail(SPADJ_ERR_INVALID, "resolvent: NULL array");
  return spadj::cou_resolvent(p->impl, p, omega, n_iter, f, gains);
}

spadj_status spadj_set_dt_schedule(spadj_problem* p, int n, const double* dts) {
  if (!p) return SPADJ_ERR_INVALID;
  if (n < 0 || (n > 0 && bad_ptr(dts))) return p->fail(SPADJ_ERR_INVALID, "set_dt_schedule: need n >= 0 and dts");
  if (p->desc.eq == SPADJ_BURGERS1D) return spadj::burgers_set_dt_schedule(p->impl, p, n, dts);
  return spadj::rb_set_dt_schedule(p->impl, p, n, dts);
}

spadj_status spadj_eigen(spadj_problem* p, int n_pencils, const double* pencil_params, const double* shifts,
                         int n_iter, double* x, double* psi, double* out) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(pencil_params) || bad_ptr(shifts) || bad_ptr(x) || bad_ptr(psi) || bad_ptr(out))
    return p->fail(SPADJ_ERR_INVALID, "eigen: NULL array");
  return spadj::evp_eigen(p->impl, p, n_pencils, pencil_params, shifts, n_iter, x, psi, out);
}

spadj_status spadj_vjp(spadj_problem* p, const double* x0, int n_steps, int ckpt_slots, int n_seeds,
                       const int* seed_steps, const double* seeds, double* grad_x0) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(x0) || bad_ptr(grad_x0) || (n_seeds > 0 && (bad_ptr(seed_steps) || bad_ptr(seeds))))
    return p->fail(SPADJ_ERR_INVALID, "vjp: NULL array");
  if (n_steps < 1 || n_seeds < 0) return p->fail(SPADJ_ERR_INVALID, "vjp: need n_steps >= 1 and n_seeds >= 0");
  std::vector<int> seed_at((size_t)n_steps + 1, -1);
  for (int i = 0; i < n_seeds; ++i) {
    const int n = seed_steps[i];
    if (n < 0 || n > n_steps) return p->fail(SPADJ_ERR_INVALID, "vjp: seed step outside 0..n_steps");
    if (seed_at[n] >= 0) return p->fail(SPADJ_ERR_INVALID, "vjp: repeated seed step");
    seed_at[n] = i;
  }
  return p->impl->vjp(p, x0, n_steps, ckpt_slots, seed_at, seeds, grad_x0);
}

spadj_status spadj_set_observations(spadj_problem* p, int n_obs, const int* obs_steps, const double* obs, int kmax) {
  if (!p) return SPADJ_ERR_INVALID;
  return spadj::kol_set_observations(p->impl, p, n_obs, obs_steps, obs, kmax);
}

spadj_status spadj_set_option(spadj_problem* p, int option, int value) {
  if (!p) return SPADJ_ERR_INVALID;
  if (option == 6) {
    p->pdl = value != 0;
    return SPADJ_OK;
  }
  if (option == 7) {
    p->fuse_columns = value != 0;
    return SPADJ_OK;
  }
  if (option == 8) {
    if (value != 1 && value != 2 && value != 4) return p->fail(SPADJ_ERR_INVALID, "set_option 8: rows per CTA must be 1, 2 or 4");
    p->x_rows = value;
    return SPADJ_OK;
  }
  if (option == 10) {
    p->bulk_staging = value != 0;
    return SPADJ_OK;
  }
  if (option == 12) {
    if (value < -1 || value > 1) return p->fail(SPADJ_ERR_INVALID, "set_option 12: -1, 0 or 1");
    p->cou_band = value;
    return SPADJ_OK;
  }
  if (option == 9) {
    if (value < 0) return p->fail(SPADJ_ERR_INVALID, "set_option 9: host checkpoint slots must be >= 0");
    p->host_slots = value;
    return SPADJ_OK;
  }
  return spadj::kol_set_option(p->impl, p, option, value);
}

spadj_status spadj_set_params(spadj_problem* p, const double* params) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(params)) return p->fail(SPADJ_ERR_INVALID, "set_params: NULL array");
  return spadj::kol_set_params(p->impl, p, params);
}

spadj_status spadj_restrict(spadj_problem* p, int n_fine, const double* fine, double* coarse) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(fine) || bad_ptr(coarse)) return p->fail(SPADJ_ERR_INVALID, "restrict: NULL array");
  return spadj::kol_restrict(p->impl, p, n_fine, fine, coarse);
}

spadj_status spadj_adam(spadj_problem* p, const double* grad_p, int t, double lr, double b1, double b2, double eps,
                        double* m, double* v, double* params) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(grad_p) || bad_ptr(m) || bad_ptr(v) || bad_ptr(params)) return p->fail(SPADJ_ERR_INVALID, "adam: NULL array");
  return spadj::kol_adam(p->impl, p, grad_p, t, lr, b1, b2, eps, m, v, params);
}

spadj_status spadj_closure_conv(spadj_problem* p, int layer, int mode, const void* in, float* out) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(in) || bad_ptr(out)) return p->fail(SPADJ_ERR_INVALID, "closure_conv: NULL array");
  return spadj::kol_closure_conv(p->impl, p, layer, mode, in, out);
}

spadj_status spadj_autotune(spadj_problem* p) {
  if (!p) return SPADJ_ERR_INVALID;
  return spadj::kol_autotune(p->impl, p);
}

spadj_status spadj_checkpoint_schedule(int n_steps, int slots, int* ops, int max_ops, int* n_ops) {
  if (n_steps < 1 || slots < 1 || !n_ops) {
    g_create_error = "checkpoint_schedule: need n_steps >= 1, slots >= 1, n_ops != NULL";
    return SPADJ_ERR_INVALID;
  }
  spadj::CkptPlanner planner;
  std::vector<spadj::CkptOp> plan = planner.plan(n_steps, slots > n_steps + 1 ? n_steps + 1 : slots);
  *n_ops = (int)plan.size();
  if (!ops) return SPADJ_OK;
  if ((int)plan.size() > max_ops) {
    g_create_error = "checkpoint_schedule: max_ops too small";
    return SPADJ_ERR_INVALID;
  }
  for (size_t i = 0; i < plan.size(); ++i) {
    ops[4 * i + 0] = plan[i].type;
    ops[4 * i + 1] = plan[i].a;
    ops[4 * i + 2] = plan[i].b;
    ops[4 * i + 3] = plan[i].slot;
  }
  return SPADJ_OK;
}

spadj_status spadj_checkpoint_schedule_host(int n_steps, int slots, int host_slots, int* ops, int max_ops,
                                           int* n_ops) {
  if (n_steps < 1 || slots < 1 || host_slots < 1 || !n_ops) {
    g_create_error = "checkpoint_schedule_host: need n_steps >= 1, slots >= 1, host_slots >= 1, n_ops != NULL";
    return SPADJ_ERR_INVALID;
  }
  spadj::CkptPlanner planner;
  std::vector<spadj::CkptOp> plan = planner.plan2(n_steps, slots, host_slots);
  *n_ops = (int)plan.size();
  if (!ops) return SPADJ_OK;
  if ((int)plan.size() > max_ops) {
    g_create_error = "checkpoint_schedule_host: max_ops too small";
    return SPADJ_ERR_INVALID;
  }
  for (size_t i = 0; i < plan.size(); ++i) {
    ops[4 * i + 0] = plan[i].type;
    ops[4 * i + 1] = plan[i].a;
    ops[4 * i + 2] = plan[i].b;
    ops[4 * i + 3] = plan[i].slot;
  }
  return SPADJ_OK;
}

spadj_status spadj_forward(spadj_problem* p, int n_steps, const double* x0, double* x_out, double* traj) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(x0) || bad_ptr(x_out)) return p->fail(SPADJ_ERR_INVALID, "forward: NULL array");
  return p->impl->forward(p, n_steps, x0, x_out, traj);
}

spadj_status spadj_tangent(spadj_problem* p, int n_steps, const double* x0, const double* dx0, double* dx_out) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(x0) || bad_ptr(dx0) || bad_ptr(dx_out)) return p->fail(SPADJ_ERR_INVALID, "tangent: NULL array");
  return p->impl->tangent(p, n_steps, x0, dx0, dx_out);
}

spadj_status spadj_adjoint(spadj_problem* p, int n_steps, const double* traj, const double* y_final,
                           double* grad_x0, double* grad_p) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(traj) || bad_ptr(y_final) || bad_ptr(grad_x0))
    return p->fail(SPADJ_ERR_INVALID, "adjoint: NULL array");
  return p->impl->adjoint(p, n_steps, traj, y_final, grad_x0, grad_p);
}

spadj_status spadj_step_forward(spadj_problem* p, int n, const double* s_n, double* s_np1) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(s_n) || bad_ptr(s_np1)) return p->fail(SPADJ_ERR_INVALID, "step_forward: NULL array");
  if (s_n == s_np1) return p->fail(SPADJ_ERR_INVALID, "step_forward: s_n and s_np1 must not be the same array");
  return p->impl->step_forward(p, n, s_n, s_np1);
}

spadj_status spadj_step_tangent(spadj_problem* p, int n, const double* s_n, const double* ds_n, double* ds_np1) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(s_n) || bad_ptr(ds_n) || bad_ptr(ds_np1)) return p->fail(SPADJ_ERR_INVALID, "step_tangent: NULL array");
  if (ds_n == ds_np1) return p->fail(SPADJ_ERR_INVALID, "step_tangent: ds_n and ds_np1 must not be the same array");
  return p->impl->step_tangent(p, n, s_n, ds_n, ds_np1);
}

spadj_status spadj_step_adjoint(spadj_problem* p, int n, const double* x_n, const double* y_np1, const double* src,
                                double* y_n, double* gp_accum) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(x_n) || bad_ptr(y_n)) return p->fail(SPADJ_ERR_INVALID, "step_adjoint: NULL array");
  if (y_np1 == y_n) return p->fail(SPADJ_ERR_INVALID, "step_adjoint: y_np1 and y_n must not be the same array");
  return p->impl->step_adjoint(p, n, x_n, y_np1, src, y_n, gp_accum);
}

spadj_status spadj_objective(spadj_problem* p, int objective, const double* obj_data, const double* x,
                             double* J_dev, double* seed) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(x) || bad_ptr(J_dev) || bad_ptr(seed)) return p->fail(SPADJ_ERR_INVALID, "objective: NULL array");
  return p->impl->objective(p, objective, obj_data, x, J_dev, seed);
}

spadj_status spadj_gradient(spadj_problem* p, const double* x0, int n_steps, int objective,
                            const double* obj_data, int ckpt_slots, double* J_host, double* grad_x0,
                            double* grad_p) {
  if (!p) return SPADJ_ERR_INVALID;
  if (bad_ptr(x0) || bad_ptr(grad_x0)) return p->fail(SPADJ_ERR_INVALID, "gradient: NULL array");
  return p->impl->gradient(p, x0, n_steps, objective, obj_data, ckpt_slots, J_host, grad_x0, grad_p);
}

spadj_status spadj_timing(spadj_problem* p, int enable) {
  if (!p) return SPADJ_ERR_INVALID;
  SPADJ_CUDA_TRY(p, cudaStreamSynchronize(p->stream));
  p->timing.reset();
  p->timing.enabled = enable != 0;
  return SPADJ_OK;
}

spadj_status spadj_timing_report(spadj_problem* p, int kernel_class, double* ms, double* flops, long* launches) {
  if (!p) return SPADJ_ERR_INVALID;
  if (kernel_class < 0 || kernel_class >= spadj::KC_COUNT || !ms || !flops || !launches)
    return p->fail(SPADJ_ERR_INVALID, "timing_report: bad kernel class or NULL output");
  p->timing.collect();
  *ms = p->timing.ms[kernel_class];
  *flops = p->timing.flops[kernel_class];
  *launches = p->timing.launches[kernel_class];
  return SPADJ_OK;
}

spadj_status spadj_couette_pencil_solve_host(int n_z, double alpha, double beta, double re, double a0, int base,
                                             int transpose, const double* in, double* out) {
  if (n_z < 8 || n_z % 4 != 0 || n_z > 128 || !(re > 0) || !(a0 > 0) || (base != 0 && base != 1) || bad_ptr(in) ||
      bad_ptr(out) || alpha < 0 || beta < 0) {
    g_create_error = "couette_pencil_solve_host: n_z a multiple of 4 in 8..128, re > 0, a0 > 0, base 0 or 1, "
                     "alpha, beta >= 0 and non-NULL arrays";
    return SPADJ_ERR_INVALID;
  }
  try {
    const spadj::rbhost::Operators o = spadj::rbhost::build_operators(n_z, 3 * n_z / 2, 1.0);
    std::string err;
    if (!spadj::couhost::band_solve_host(o, alpha, beta, 1.0 / re, a0, base, transpose != 0,
                                         reinterpret_cast<const std::complex<double>*>(in),
                                         reinterpret_cast<std::complex<double>*>(out), &err)) {
      g_create_error = err;
      return SPADJ_ERR_INVALID;
    }
  } catch (const std::bad_alloc&) {
    return SPADJ_ERR_NOMEM;
  }
  return SPADJ_OK;
}

const char* spadj_last_error(const spadj_problem* p) {
  if (!p) return g_create_error.c_str();
  return p->err.empty() ? "no error" : p->err.c_str();
}

}  // extern "C"
