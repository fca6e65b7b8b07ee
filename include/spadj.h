/*
 * spadj.h -- C-ABI of the GB300 library for IMEX spectral timesteps and their exact
 * discrete adjoints (arXiv 2506.14792, "Fast automated adjoints for spectral PDE solvers").
 *
 * The library implements, in hand-written CUDA for sm_103a, one IMEX timestep of a
 * sparse spectral discretisation of  M dX/dt + L X = F(X, p)  (Supplementary A.4) and
 * the adjoint of that step run backward over a checkpointed trajectory, and the
 * gradient of an objective J with respect to the initial condition
 * (eqs. 1-6, "Efficiently calculating gradients").
 *
 * Conventions (all entry points):
 *  - Every array argument is caller-owned DEVICE memory (for example from torch), read
 *    and written on the problem's CUDA stream, unless the name ends in _host.
 *  - Coefficient arrays are float64 and hold complex coefficients as interleaved
 *    (re, im) pairs; the layout of each equation set is given at spadj_eq below.
 *    The inner product that defines every adjoint is the Euclidean one over these
 *    stored reals (the paper's "suitably chosen inner product", Continuous vs.
 *    discrete section).
 *  - Calls are asynchronous on the stream except where a _host output is written
 *    (then the call synchronises the stream before returning).
 *  - The library owns its factorisations, workspaces and checkpoint slots; it
 *    allocates them in spadj_create or lazily on first use, and frees them in
 *    spadj_destroy.
 *  - Every call returns a spadj_status; on failure spadj_last_error() gives a
 *    one-line reason.  No call falls back to CPU arithmetic.
 */
#ifndef SPADJ_H
#define SPADJ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spadj_problem spadj_problem; /* opaque, library-owned */

typedef enum {
  SPADJ_OK = 0,
  SPADJ_ERR_INVALID = -1,     /* bad descriptor, size or pointer */
  SPADJ_ERR_NOMEM = -2,       /* device allocation failed or checkpoint budget too small */
  SPADJ_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  SPADJ_ERR_NONFINITE = -4,   /* a NaN/Inf was detected in the state or objective */
  SPADJ_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
  SPADJ_ERR_UNSUPPORTED = -6  /* operation not defined for this equation/scheme */
} spadj_status;

/*
 * Equation sets and their coefficient layouts (B = batch size from the descriptor).
 *
 * SPADJ_BURGERS1D: u_t - nu u_xx = -d/dx(u^2/2) on [0, length[0]), periodic Fourier
 *   basis, N = n[0] modes, 3/2-dealiased grid of 3N/2 points.  State per member:
 *   K = N/2 complex coefficients c_k (k = 0..K-1; Nyquist not stored; Im c_0 held at 0).
 *   Layout [B][K] complex.  Grid layout [B][3N/2] real.  params[0] = nu.
 *
 * SPADJ_RB2D: Boussinesq convection in free-fall units, buoyancy b = 1 - z + theta,
 *   x in [0, length[0]) periodic Fourier (Nx = n[0] modes), z in [0, 1] Chebyshev-T
 *   (N = n[1] modes) with tau terms; equations projected on the ultraspherical C^(2)
 *   (momentum, temperature) and C^(1) (continuity) bases, no-slip, fixed temperature
 *   (Sparse spectral methods section).  params[0] = Ra, params[1] = Pr (nu = (Ra/Pr)^-1/2,
 *   kappa = (Ra Pr)^-1/2).  Scheme RK222 (or RK443).  State: u, w, theta coefficients, layout
 *   [3][Nx/2][N] complex (x-mode m = 0..Nx/2-1, Nyquist not stored; the m = 0 pencil is
 *   held real).  Grid layout [3N/2][3Nx/2] real (Gauss-Chebyshev z rows, uniform x).
 *   Pressure and tau variables are internal to the stage solves.
 *
 * SPADJ_KOLMOGOROV2D: 2D vorticity d_t w - lap w / Re = -(u d_x w + v d_y w) - 4 cos 4y on
 *   [0, 2 pi)^2 (body force sin(4y) e_x), u = d_y psi, v = -d_x psi, lap psi = -w; Fourier
 *   in x and y, 3/2 dealiasing; SBDF1 then SBDF2.  params[0] = Re, params[1] = 1 to drop the
 *   forcing (tests).  A batch may mix resolutions (desc.batch_n).  Member b with N_b modes
 *   holds N_b/2 x N_b complex coefficients, layout [kx][ky] (kx = 0..N/2-1, ky index j holds
 *   ky = j for j < N/2 and j - N otherwise; the ky = -N/2 row is held at 0 and the kx = 0
 *   column Hermitian); members are concatenated in batch order.  All members advance in one
 *   persistent launch over (stage, phase, member, tile) work items.
 *
 * SPADJ_COUETTE3D: perturbation u = (u, v, w) of plane Couette flow U = z between walls at
 *   z = -1, +1 moving with -1, +1:  dt u - lap u / Re + U dx u + w U' e_x + grad p = u x curl u,
 *   div u = 0, no-slip (p is the dynamic pressure).  x in [0, length[0]) (default 4 pi) and
 *   y in [0, length[1]) (default 2 pi) periodic Fourier (Nx = n[0], Ny = n[1] modes), z
 *   Chebyshev-T (N = n[2] modes) with tau terms as for SPADJ_RB2D; 3/2 dealiasing on all axes.
 *   params[0] = Re; params[1] = laminar profile: 0 (default) plane Couette U = z as above,
 *   1 plane Poiseuille (channel) flow U = 1 - z^2 between stationary walls (the profile of the
 *   Parametric sensitivity example; its driving pressure gradient is held fixed).  Scheme SBDF2
 *   (SBDF1 first step).  State: u, v, w coefficients, layout
 *   [3][Ny][Nx/2][N] complex (ky index j in FFT order as for SPADJ_KOLMOGOROV2D, kx index
 *   m = 0..Nx/2-1 with the Nyquist not stored; the ky = -Ny/2 row is held at 0 and the kx = 0
 *   plane Hermitian in ky).  Grid layout [3N/2][3Ny/2][3Nx/2] real (Gauss-Chebyshev z).
 *   Pressure and tau variables are internal to the step solves.
 *
 * SPADJ_SHEAR_EVP: linear stability eigenproblems (lambda M + L) X = 0 of plane shear flows
 *   (Problem types, "Eigenvalue problems"; Parametric sensitivity example): perturbations
 *   exp(i (alpha x + beta y) + lambda t) of the laminar profile U(z) e_x between no-slip walls
 *   at z = -1, +1, lambda u - lap u / Re + U dx u + w U' e_x + grad p = 0, div u = 0, with the
 *   z discretisation of SPADJ_COUETTE3D (N = n[2] Chebyshev modes, 8 <= N <= 128).
 *   params[0] = base flow: 0 = plane Couette U = z, 1 = plane Poiseuille U = 1 - z^2 (the
 *   paper's y (2 - y) on [0, 2] in z = y - 1; Re on the centre-line velocity and half gap).
 *   batch = the largest number of pencils per spadj_eigen call; dt, scheme and the other
 *   fields are unused.  Vectors: [n_pencils][3N] complex, the Chebyshev-T coefficients of
 *   u, v, w of a pencil (pressure and tau variables are internal).
 */
typedef enum {
  SPADJ_BURGERS1D = 0,
  SPADJ_RB2D = 1,
  SPADJ_KOLMOGOROV2D = 2,
  SPADJ_COUETTE3D = 3,
  SPADJ_SHEAR_EVP = 4
} spadj_eq;

typedef enum {
  SPADJ_SBDF1 = 1, /* multistep IMEX, eq. imex, first order */
  SPADJ_SBDF2 = 2, /* multistep IMEX, eq. imex, second order (SBDF1 first step) */
  SPADJ_RK222 = 3, /* Runge-Kutta IMEX ARS(2,2,2), Supplementary A.4 stage equation */
  SPADJ_SBDF3 = 4, /* multistep IMEX, third order (SPADJ_BURGERS1D; SBDF1, SBDF2 first steps) */
  SPADJ_SBDF4 = 5, /* multistep IMEX, fourth order (SPADJ_BURGERS1D; SBDF1..3 first steps) */
  SPADJ_RK443 = 6  /* Runge-Kutta IMEX ARS(4,4,3), third order (SPADJ_RB2D; separate kernels) */
} spadj_scheme;

typedef struct {
  int eq;            /* spadj_eq */
  int scheme;        /* spadj_scheme */
  int n[3];          /* modes per axis (unused axes 0) */
  double length[3];  /* domain lengths per axis */
  double params[4];  /* equation parameters (see spadj_eq) */
  double dt;         /* constant timestep */
  int batch;         /* number of independent members advanced together (>= 1) */
  int nonlinear;     /* 1: F as defined; 0: F = 0 (linear problem, used by tests) */
  const int* batch_n;/* host, nullable: per-member resolution of a mixed batch (SPADJ_KOLMOGOROV2D);
                        NULL = every member uses n[0].  Copied by spadj_create. */
  int closure;       /* SPADJ_KOLMOGOROV2D: 1 adds the learned CNN closure C(w; p) to F on the grid
                        (uniform resolution; parameters set by spadj_set_params, initially 0) */
} spadj_desc;

/* Build a problem (operators, transform tables, factorisations) bound to cuda_stream
 * (a cudaStream_t; NULL = legacy default stream).  *out receives the handle. */
spadj_status spadj_create(const spadj_desc* desc, void* cuda_stream, spadj_problem** out);

/* Free everything the problem owns.  Synchronises the stream first. */
spadj_status spadj_destroy(spadj_problem* prob);

/* Lengths in float64 elements for the whole batch:
 * which = 0: coefficient state (the vector the gradient is taken with respect to);
 * which = 1: one real grid field;  which = 2: parameter vector p;
 * which = 3: one scalar coefficient field (the input/output of spadj_transform);
 * which = 4: restart state of one step (spadj_step_forward / spadj_step_tangent);
 * which = 5: adjoint state of one step (spadj_step_adjoint).
 * 4 and 5 are 0 where the step entry points are not provided. */
size_t spadj_state_len(const spadj_problem* prob, int which);

/* Collocation transforms (Methods, "Spectral transforms"): kind
 *  0 = c2g  (T^-1: coefficients -> grid),      1 = g2c  (T: grid -> coefficients),
 *  2 = c2g adjoint (T^-dagger... applied as (T^-1)^dagger: grid -> coefficients),
 *  3 = g2c adjoint (T^dagger: coefficients -> grid).
 * in/out are device arrays in the coefficient or grid layout of the equation set. */
spadj_status spadj_transform(spadj_problem* prob, int kind, const double* in, double* out);

/* spadj_transform without any device allocation, for callers that cannot call cudaMalloc:
 * processes whose device memory is owned by their own allocator (a framework's caching
 * allocator or an arena reserved at start-up) and may not go around it, and latency-bound
 * loops that cannot afford cudaMalloc/cudaFree, which can synchronise the device.  The paper
 * has no counterpart; this is an interface convenience of this library.
 * Defined for SPADJ_RB2D only (SPADJ_ERR_UNSUPPORTED otherwise).  Same kinds, layouts and
 * results as spadj_transform.  Its intermediate array (3*n[1]/2 x n[0]/2 complex entries)
 * lives in a static device array of 262144 complex entries (4 MiB) that every GPU loading
 * the library holds until the process exits; larger sizes return SPADJ_ERR_INVALID.  The
 * first call on a device looks the array's address up (cudaGetSymbolAddress, with the
 * problem's device current); make that first call before any stream capture.  All calls
 * share the one array: calls whose kernels overlap on the GPU (different streams, or
 * different problems on one device) race and must be serialised by the caller.  The array
 * is fully overwritten before it is read, so no clearing is needed between calls. */
spadj_status spadj_transform_noalloc(spadj_problem* prob, int kind, const double* in, double* out);

/* Explicit term F(X) in coefficient space (Sparse spectral methods section: nonlinear
 * terms evaluated on the dealiased collocation grid), its Jacobian-vector product
 * dF = (dF/dX) dX and its vector-Jacobian product out = (dF/dX)^dagger y
 * (Methods, "Nonlinear operator graphs"). */
spadj_status spadj_eval_F(spadj_problem* prob, const double* x, double* f);
spadj_status spadj_eval_F_jvp(spadj_problem* prob, const double* x, const double* dx, double* df);
spadj_status spadj_eval_F_vjp(spadj_problem* prob, const double* x, const double* y, double* out);

/* Stage solve of the sparse pencil systems (Methods, "Linear system solves"), defined for
 * SPADJ_RB2D: x = prognostic part of (M + dt*gamma*L)^-1 [S1S0 v; 0] per x-mode pencil, and
 * for SPADJ_COUETTE3D: x = P (prognostic part of ((3/(2 dt)) M + L)^-1 [S1S0 v; 0]) per
 * (kx, ky) pencil (the SBDF2 step matrix; P the projection onto admissible coefficients),
 * v and x in the state layout (T coefficients).  transpose = 1 applies the adjoint map
 * (Hermitian transpose, reusing the same factorisation).  SPADJ_ERR_UNSUPPORTED otherwise. */
spadj_status spadj_solve(spadj_problem* prob, int transpose, const double* v, double* x);

/* Binomial checkpoint schedule used by spadj_gradient (host only, no GPU needed): for
 * n_steps steps and `slots` state slots (slot 0 = initial state) writes n_ops actions of
 * 4 ints (type, a, b, slot) to ops (host) if ops != NULL and max_ops suffices.  Types:
 * 0 advance a->b, 1 store state a in slot, 2 restore state a from slot, 3 adjoint of step a
 * (state X_a current), 4 free slot, 5 evaluate the objective at state a. */
spadj_status spadj_checkpoint_schedule(int n_steps, int slots, int* ops, int max_ops, int* n_ops);

/* Two-level schedule used by spadj_gradient / spadj_vjp when host checkpoint slots are set
 * (spadj_set_option 9, SPADJ_RB2D and SPADJ_COUETTE3D): the first forward sweep stores X_a in
 * host memory at the start of every segment [a, a + K), K = ceil(n_steps / host_slots), and the
 * segments are reversed last first, each from its host copy by the binomial schedule on the
 * `slots` device slots (the paper's RAM + disk checkpointing, after H-revolve).  Same action
 * encoding as spadj_checkpoint_schedule; host slots are numbered slots .. slots + host_slots - 1. */
spadj_status spadj_checkpoint_schedule_host(int n_steps, int slots, int host_slots, int* ops, int max_ops,
                                           int* n_ops);

/* Forward trajectory of n_steps IMEX steps from x0 (eq. imex / RK stage equation).
 * x_out receives X_N.  traj (nullable) receives X_0..X_N, layout [n_steps+1][state]. */
spadj_status spadj_forward(spadj_problem* prob, int n_steps, const double* x0, double* x_out,
                           double* traj);

/* Tangent (JVP) trajectory: dx_out = dX_N for the perturbation dx0 of x0. */
spadj_status spadj_tangent(spadj_problem* prob, int n_steps, const double* x0, const double* dx0,
                           double* dx_out);

/* Adjoint sweep over a stored trajectory traj (= X_0..X_N from spadj_forward):
 * seeds the cotangent y_final = dJ/dX_N and returns grad_x0 = dJ/dX_0 by the
 * discrete adjoint recurrence (eq. IMEX_adjoint / RK adjoint, Supplementary A.4).
 * grad_p (device, nullable; spadj_state_len(prob, 2) values) receives the parameter
 * gradient sum_n (dF(X_n)/dp)^dagger (sum_i c_i^{n+i} Y_{n+i}) (eq. 6 with p entering F); it
 * must be NULL for problems without parameters (SPADJ_ERR_INVALID / SPADJ_ERR_UNSUPPORTED). */
spadj_status spadj_adjoint(spadj_problem* prob, int n_steps, const double* traj,
                           const double* y_final, double* grad_x0, double* grad_p);

/* One timestep at a time: the forward step, its tangent and its adjoint as separate calls, so a
 * caller can drive its own schedule (the problem statement's "step forward" and "step adjoint";
 * eq. imex / the RK stage equation and their adjoints eq. IMEX_adjoint / RK adjoint,
 * Supplementary A.4; eqs. 5-6, "Efficiently calculating gradients").  Defined for SPADJ_RB2D
 * (RK222, RK443), SPADJ_COUETTE3D (SBDF1, SBDF2), SPADJ_BURGERS1D (SBDF1-4) and SPADJ_KOLMOGOROV2D
 * (SBDF2; forward and adjoint steps, no tangent; with the closure the adjoint step adds the step's
 * parameter cotangent to gp_accum); other equation sets return SPADJ_ERR_UNSUPPORTED.  Step n (n >= 0) maps X_n to X_{n+1}; with a step-size
 * schedule it uses dts[n], and a multistep scheme of order s uses order min(n + 1, s) as the
 * sweeps do.  All arrays are caller-owned device memory on the problem's stream; input and output
 * arrays must be distinct.  Chained from X_0, the forward and adjoint steps reproduce the sweeps
 * (spadj_forward, spadj_gradient, spadj_vjp) bit for bit: the same kernels run on the same data;
 * so does the tangent (spadj_tangent), except for SPADJ_RB2D with RK222, whose tangent sweep
 * recomputes the primal stages with the unfused column kernels (agreement to rounding).
 *
 * Restart state s_n (spadj_state_len(prob, 4) doubles): the data step n needs.
 *   Runge-Kutta: X_n.
 *   Multistep of order s: blocks of one state each,
 *   [X_n, X_{n-1}, ..., X_{n-s+1}, F(X_{n-1}), ..., F(X_{n-s+1})] (2s - 1 blocks); blocks that do
 *   not exist yet (n < s - 1) are not read by the lower-order first steps.  For n = 0 set X_0 and
 *   zeros.
 * spadj_step_forward writes s_{n+1}; spadj_step_tangent writes ds_{n+1}, the tangent (JVP) of
 * s_{n+1} along ds_n (same layout), for the primal restart state s_n. */
spadj_status spadj_step_forward(spadj_problem* prob, int n, const double* s_n, double* s_np1);
spadj_status spadj_step_tangent(spadj_problem* prob, int n, const double* s_n, const double* ds_n,
                                double* ds_np1);

/* Adjoint of step n.  Adjoint state y (spadj_state_len(prob, 5) doubles):
 *   Runge-Kutta: y_n = Y_n, the cotangent of X_n: y_n = (dX_{n+1}/dX_n)^dagger y_{n+1} + src.
 *   Multistep of order s: y_n = [Y_n, Y_{n+1}, ..., Y_{n+s-1}], the adjoint variables of
 *   eq. IMEX_adjoint (for SPADJ_COUETTE3D in prognostic form): the right-hand side
 *   R_n = sum_{i=1..s} (c_i^{n+i} dF/dX(X_n) - a_i^{n+i} M - b_i^{n+i} L)^dagger Y_{n+i} + src is
 *   formed and, for n >= 1, (a_0^n M + b_0^n L)^dagger Y_n = R_n solved; for n = 0 the first block
 *   of y_0 is R_0 = dJ/dX_0 (the gradient with respect to the initial state: no solve).
 * x_n: the primal state X_n (one state, not the restart state).  y_np1 = NULL stands for zero
 * adjoint variables.  src (nullable) is dJ/dX_n, the objective's explicit dependence on X_n.
 * The chain that gives dJ/dX_0 is the same for every scheme:
 *   y = NULL;  for n = N, N-1, ..., 0:  y = step_adjoint(n, X_n, y, dJ/dX_n);  dJ/dX_0 = y[0 : state]
 * (at n = N a Runge-Kutta step returns src; a multistep step solves for Y_N).
 * gp_accum (nullable): for problems with parameters (SPADJ_KOLMOGOROV2D with the learned closure),
 * the step's parameter cotangent (dF(X_n)/dp)^dagger (sum_i c_i^{n+i} Y_{n+i}) is added to it
 * (spadj_state_len(prob, 2) doubles), so the chain accumulates dJ/dp; problems without parameters
 * require NULL and return SPADJ_ERR_INVALID otherwise. */
spadj_status spadj_step_adjoint(spadj_problem* prob, int n, const double* x_n, const double* y_np1,
                                const double* src, double* y_n, double* gp_accum);

/* Objectives for spadj_gradient. */
typedef enum {
  SPADJ_OBJ_ENERGY = 0,   /* J = 1/2 ||u(T)||^2 (physical L2 integral) per batch member; for
                             SPADJ_COUETTE3D J = E(X_N) = (1/V) int |u|^2 dV */
  SPADJ_OBJ_FOURDVAR = 1, /* J = sum_m 1/2 ||H(X_{n_m}) - obs_m||^2 per member (observations set by
                             spadj_set_observations; H keeps |kx|, |ky| <= kmax) */
  SPADJ_OBJ_GAIN = 2,     /* SPADJ_COUETTE3D: energy gain J = E(X_N) / E(X_0) with the
                             volume-weighted norm E(X) = (1/V) int |u|^2 dV (optimal
                             perturbation objective); spadj_objective takes X_0 as obj_data
                             and returns dJ/dX_N only, spadj_gradient includes the explicit
                             dependence on X_0 */
  SPADJ_OBJ_ENERGY_INTEGRAL = 3 /* SPADJ_COUETTE3D, spadj_gradient only: J = I(T) with
                             dI/dt = E(X), I(0) = 0, the ODE added to the equation set and
                             integrated by the same IMEX scheme (Supplementary A.4), so the
                             time integral has the scheme's accuracy and its cotangents enter
                             the adjoint sweep at every step */
} spadj_objective_kind;

/* 4D-Var observations for SPADJ_OBJ_FOURDVAR (SPADJ_KOLMOGOROV2D): n_obs steps (host ints,
 * increasing, in 1..n_steps of the later gradient call), obs (device, layout [n_obs][state],
 * copied by the call) and the low-pass cut-off kmax of the observation operator H. */
spadj_status spadj_set_observations(spadj_problem* prob, int n_obs, const int* obs_steps, const double* obs,
                                    int kmax);

/* Parameters p of the learned closure (device, spadj_state_len(prob, 2) float64 values: per
 * layer the 3x3 weights W[o][c][a][b] then the biases; channels 1 -> 32 -> 32 -> 32 -> 1, tanh
 * after the first three layers, periodic padding).  The network runs with BF16 operands and
 * FP32 accumulation; spadj_gradient's grad_p receives dJ/dp (eq. 6 with p entering F). */
spadj_status spadj_set_params(spadj_problem* prob, const double* params);

/* Training support for the learned closure (the paper names coupling the adjoints to learned
 * models as future work, Conclusions; these two calls are not part of its method).
 * spadj_restrict: spectral truncation R of B fine members to the resolution of prob, a
 * SPADJ_KOLMOGOROV2D problem of uniform resolution Nc = n[0] and batch B: coarse (kx, ky) = fine
 * (kx, ky) for kx < Nc/2 and |ky| < Nc/2, the coarse ky = -Nc/2 row zero.  fine (device): B members
 * of n_fine >= Nc modes each ([B][n_fine/2][n_fine] complex, the layout of SPADJ_KOLMOGOROV2D);
 * coarse (device): spadj_state_len(prob, 0) doubles.  SPADJ_ERR_INVALID for an odd or too small
 * n_fine, SPADJ_ERR_UNSUPPORTED for a mixed-resolution batch.
 * spadj_adam: one Adam step (Kingma & Ba, 2015) on the closure parameters: with g = grad_p,
 * m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2, params <- params - lr mhat / (sqrt(vhat) + eps),
 * mhat = m / (1 - b1^t), vhat = v / (1 - b2^t); t >= 1 is the step count.  grad_p, m, v, params:
 * device arrays of spadj_state_len(prob, 2) doubles, m and v owned by the caller (zero before the
 * first step).  The parameters of the problem are not changed: call spadj_set_params. */
spadj_status spadj_restrict(spadj_problem* prob, int n_fine, const double* fine, double* coarse);

/* Test support for the learned closure's tensor-core kernels (not part of the method): one 32 -> 32
 * convolution of hidden layer `layer` (1 or 2) with the problem's current BF16 weights (spadj_set_params)
 * over all batch members of its M x M grid (M = 3 n[0] / 2): mode 0 the pre-activation
 * out = conv(in) + b (forward), mode 1 the input gradient out = conv^T(in) (no bias), mode 2 the
 * derivative of the activation the forward epilogue stores, out = 1 - tanh(conv(in) + b)^2 (the
 * layer's BF16 activations are overwritten in the problem's own buffer).  in: device, BF16
 * bit patterns, [member][y][x][32 channels]; out: device float32, same layout.  Runs the kernel the
 * closure passes use (tcgen05 MMAs with the accumulator in tensor memory, unless spadj_set_option 11
 * selected the mma.sync kernel, which has no mode 0 here).  Synchronises the stream;
 * SPADJ_ERR_TIMEOUT if a bounded wait for the MMAs ran out. */
spadj_status spadj_closure_conv(spadj_problem* prob, int layer, int mode, const void* in, float* out);
spadj_status spadj_adam(spadj_problem* prob, const double* grad_p, int t, double lr, double b1, double b2,
                        double eps, double* m, double* v, double* params);

/* Tuning knobs of the batched persistent launch (SPADJ_KOLMOGOROV2D): option 0 = persistent
 * scheduler (1, default) or one launch per phase (0); with the closure the persistent scheduler
 * runs one launch per step (the network's whole-grid passes run between the launches) and is the
 * default only for batches of at least 64 grid rows per SM; 1 = x-modes per column tile;
 * 2 = grid rows per row tile; 3 = resident CTAs per SM (0 = occupancy maximum); 4 = iteration
 * limit of the scheduler's bounded waits (0 = default, several seconds); 5 = failure-path test:
 * the completion of this member (-1 = none) is never signalled, so a bounded wait runs out and
 * the call returns SPADJ_ERR_TIMEOUT with the context intact.  Option 6 (SPADJ_RB2D,
 * SPADJ_COUETTE3D) = programmatic dependent launch of consecutive kernels (1: the next kernel
 * is scheduled while its predecessor drains and waits for it on the device; 0, default: plain
 * stream order); option 7 (SPADJ_RB2D) = fused column stage (1, default: the z fold, the stage
 * solve and the z expansion of each x-mode pencil run in one two-CTA cluster kernel; 0: three
 * separate kernels); option 8 (SPADJ_RB2D, SPADJ_COUETTE3D) = grid rows per CTA of the x FFTs
 * (1, 2 or 4, 64 threads per CTA; by default the fastest of these and of 2 or 4 rows on 96, 128
 * or 192 threads is picked by timing when the problem is created); option 9
 * (SPADJ_RB2D, SPADJ_COUETTE3D) = host checkpoint slots of spadj_gradient / spadj_vjp (0, default:
 * device slots only; h > 0: the two-level schedule of spadj_checkpoint_schedule_host, the host
 * copies in page-locked memory owned by the problem); option 10 (SPADJ_RB2D) = how the fused column
 * stages bring their operator block into shared memory (1, default: one bulk copy, cp.async.bulk,
 * completing on an mbarrier; 0: 16-byte cp.async copies spread over the threads); option 11
 * (SPADJ_KOLMOGOROV2D with the closure) = the 32 -> 32 convolutions on the fifth-generation tensor
 * cores (tcgen05.mma, accumulator in tensor memory) with the operand staged once per tile and the
 * nine taps read through shifted descriptors (1, default), the same with the operand gathered once
 * per tap (2), or on warp-level mma.sync (0); option 13 (SPADJ_KOLMOGOROV2D with the closure) =
 * how the thin layers' (1 -> 32, 32 -> 1) weight gradients are summed (1, default: all nine taps
 * in one CTA per row band and member, the input window in registers; 0: one CTA per x offset);
 * option 14 (SPADJ_KOLMOGOROV2D with the closure) = how the thin layers' single-channel outputs
 * (the 32 -> 1 forward, the 1 -> 32 input gradient) are summed (1, default: row segments with the
 * 32-channel window in registers, channel pairs added across the half-warp; 0: one thread per
 * pixel);
 * option 12 (SPADJ_COUETTE3D) = form of the step solves (1: forward and back sweeps with the
 * banded LU factors of each recombined, mode-ordered pencil matrix, one warp per pencil pair;
 * 0: the dense prognostic operator Phi applied as a matvec; -1, default: banded when there are at
 * least 8 pencil pairs per SM, else dense; both compute the same map up to rounding, and the form
 * not built at creation is built on its first use).  Set them before the
 * first sweep (the step graphs are captured once).
 * spadj_autotune times candidate settings on the problem's own sizes and keeps the fastest. */
spadj_status spadj_set_option(spadj_problem* prob, int option, int value);
spadj_status spadj_autotune(spadj_problem* prob);

/* Objective J(X) per batch member and its partial derivative (eq. 1's dJ/dX), which seeds
 * the adjoint sweep: J_dev receives B doubles (device), seed receives dJ/dX (state layout).
 * obj_data is objective-specific (NULL for SPADJ_OBJ_ENERGY). */
spadj_status spadj_objective(spadj_problem* prob, int objective, const double* obj_data, const double* x,
                             double* J_dev, double* seed);

/* Gradient of an objective with respect to the initial condition (eqs. 1-6):
 * forward sweep with checkpoints (ckpt_slots <= 0: store every step; the schedules per equation
 * set are those of spadj_vjp), objective, adjoint sweep with recomputation.  J_host receives J per batch member (host
 * memory, B doubles); grad_x0 receives dJ/dX_0.  obj_data and grad_p may be NULL. */
spadj_status spadj_gradient(spadj_problem* prob, const double* x0, int n_steps, int objective,
                            const double* obj_data, int ckpt_slots, double* J_host,
                            double* grad_x0, double* grad_p);

/* Measurement support (not part of the method): when enabled, every kernel the library
 * launches on the problem's stream is bracketed by CUDA events; spadj_timing_report
 * returns, per kernel class, the summed device time (ms), the summed algorithmic FP64
 * flop count and the number of launches since timing was (re)enabled.  Classes:
 * 0 z (Chebyshev) transforms, 1 x (Fourier) FFTs, 2 grid-point products, 3 pencil solves,
 * 4 objective, 5 fused persistent trajectory kernels, 6 y (Fourier) FFTs, 7 energy-norm (Gram)
 * products of the resolvent iteration, 8 the learned closure's network passes (BF16 operands,
 * FP32 accumulation).  spadj_timing
 * synchronises the stream and resets the counters. */
spadj_status spadj_timing(spadj_problem* prob, int enable);
spadj_status spadj_timing_report(spadj_problem* prob, int kernel_class, double* ms, double* flops, long* launches);

/* Measurement support (not part of the method): FP64 fused-multiply-add throughput of the current
 * device, the denominator of the FP64-bound kernels' roofline fractions.  Runs a kernel of
 * independent FMA chains (iters FMAs per chain, an occupancy-sized grid) on cuda_stream, timed with
 * CUDA events after a warm-up launch; *gflops_host receives 2 x FMAs / time (GFLOP/s) and *ms_host
 * (nullable) the timed duration.  Synchronises the stream; allocates and frees a small buffer. */
spadj_status spadj_fp64_peak(void* cuda_stream, int iters, double* gflops_host, double* ms_host);

/* Test support (host only, no GPU; not part of the method): the banded step solve of one plane-
 * Couette pencil computed on the host with the factors and the sweep order the GPU kernel uses
 * (option 12 = 1), so that the factorisation can be checked against a dense solve without a GPU.
 * Pencil (kx, ky) = (alpha, beta) >= 0 of the z discretisation with n_z Chebyshev modes (a multiple
 * of 4 in 8..128), Re = re, base flow `base` (0 plane Couette, 1 plane Poiseuille), shift a0 > 0
 * (1/dt for SBDF1, 1.5/dt for SBDF2).  transpose = 0: out = [(a0 M + L)^-1 (S1S0 in on the momentum
 * rows)] restricted to the u, v, w coefficients; transpose = 1: out = S1S0^T [momentum rows of
 * (a0 M + L)^-H (in on the u, v, w rows)] (the adjoint map).  in, out: host arrays of 3 n_z complex
 * values (u, v, w blocks; interleaved re, im).  SPADJ_ERR_INVALID for bad arguments or a singular
 * pencil (spadj_last_error(NULL) says which). */
spadj_status spadj_couette_pencil_solve_host(int n_z, double alpha, double beta, double re, double a0, int base,
                                             int transpose, const double* in, double* out);

/* Vector-Jacobian product of the trajectory map (the reverse-mode building block behind
 * spadj_gradient and the torch.autograd binding): grad_x0 = sum_i (dX_{n_i}/dX_0)^T seed_i for
 * cotangents seeds[i] (device, layout [n_seeds][state]) injected at steps seed_steps[i]
 * (host ints in 0..n_steps, distinct).  Checkpointing (as in spadj_gradient): ckpt_slots <= 0 stores
 * every step; SPADJ_RB2D, SPADJ_COUETTE3D and SPADJ_BURGERS1D run the binomial schedule on ckpt_slots
 * device slots (two-level with host slots, spadj_set_option 9); SPADJ_KOLMOGOROV2D keeps the restart
 * state [X_a, X_{a-1}, F(X_{a-1})] of each of ckpt_slots segments (device memory, or page-locked host
 * memory for the option 9 count of segments), recomputes one segment's trajectory at a time and
 * reverses it in one persistent launch (the adjoint variables of eq. IMEX_adjoint carried from one
 * segment's launch to the next).  This is the
 * adjoint sweep of Supplementary A.4 with the objective's partial derivatives replaced by the
 * given cotangents (4D-Var style injection at intermediate steps included). */
spadj_status spadj_vjp(spadj_problem* prob, const double* x0, int n_steps, int ckpt_slots, int n_seeds,
                       const int* seed_steps, const double* seeds, double* grad_x0);

/* Hessian-vector product (SPADJ_COUETTE3D, objective SPADJ_OBJ_ENERGY: J = E(X_N)):
 * hv = (d^2 J / dX_0^2) v by tangent-over-adjoint: a forward sweep with its tangent along v
 * (both trajectories stored, 2 (n_steps + 1) states of device memory held by the problem),
 * then the adjoint recurrence and its tangent run together (three vector-Jacobian products and
 * two transposed pencil solves per step).  x0, v, hv: device, state layout. */
spadj_status spadj_hvp(spadj_problem* prob, const double* x0, const double* v, int n_steps, double* hv);

/* Resolvent gains of the linear operator (SPADJ_COUETTE3D): for every (kx, ky) pencil, the
 * leading gain sigma_1 = max ||R f||_E / ||f||_E of R(omega) = prognostic part of
 * (i omega M + L)^-1 [S1S0 f; 0] (the response of u, v, w to a momentum forcing f at frequency
 * omega) in the energy norm ||c||_E^2 = sum over u, v, w of c^H G c (G_mn = int T_m T_n dz),
 * by n_iter power iterations on R^H G R f = sigma^2 G f for all pencils at once, with the
 * transposed pencil solves supplying R^H (the LBVP adjoint).  f (device, state layout) is the
 * initial forcing on entry and the leading forcing (unit energy per pencil) on exit; gains
 * (device, [Ny][Nx/2] doubles) receives sigma_1 per pencil (0 where the initial forcing of the
 * pencil is zero).  The pencil factorisations of (i omega M + L) are built on the first call
 * for a frequency and kept until another frequency is asked for. */
spadj_status spadj_resolvent(spadj_problem* prob, double omega, int n_iter, double* f, double* gains);

/* Step-size schedule (SPADJ_RB2D, SPADJ_BURGERS1D): step n of every later forward, tangent, adjoint,
 * gradient, vjp and step call uses dts[n] (host array of n > 0 sizes, copied; n = 0 restores the
 * descriptor's constant dt).  SPADJ_RB2D: the stage operators M + dt gamma L are factorised once per
 * distinct size, when a sweep first needs it, and kept for later sweeps: the paper's timesteppers
 * reuse their LU factorisations unless the timestep changes, and rebuild them when it does.
 * SPADJ_BURGERS1D (SBDF1 or SBDF2; SPADJ_ERR_UNSUPPORTED for SBDF3/4): variable-step SBDF2, the
 * weights of step n from its own size h_n and the ratio w = h_n / h_{n-1} (Wang-Ruuth form:
 * a0 = (1 + 2w)/((1 + w) h_n), a1 = -(1 + w)/h_n, a2 = w^2/((1 + w) h_n), c1 = 1 + w, c2 = -w; the first
 * step SBDF1 of size h_1), the diagonal solve 1/(a0 + nu k^2) refreshed when a0 changes.  The
 * adjoint of step n uses the same weights as its forward step.  A sweep longer than the schedule
 * fails with SPADJ_ERR_INVALID; sizes must be positive.  spadj_solve keeps the descriptor's dt. */
spadj_status spadj_set_dt_schedule(spadj_problem* prob, int n, const double* dts);

/* Leading eigenvalue and its parameter sensitivities for a batch of pencils (SPADJ_SHEAR_EVP).
 * Pencil i has pencil_params[3i..3i+2] = (alpha, beta, Re) and the complex shift sigma_i =
 * shifts[2i] + i shifts[2i+1] (host arrays, read during the call).  The library factorises
 * A_i = sigma_i M + L_i on the host (one LU per pencil, the adjoint solves reuse it) and on the
 * GPU runs n_iter shift-invert power iterations on the prognostic block Phi_i of A_i^-1 M
 * (eigenvalues 1/(sigma_i - lambda)) and, in the same pass over Phi_i, on Phi_i^H (the adjoint
 * eigenproblem), so it converges to the eigenvalue nearest sigma_i.  Then, with the full right
 * and left eigenvectors X and Y ((lambda M + L) X = 0, (conj(lambda) M^H + L^H) Y = 0), the
 * sensitivities of eq. eigenvalue_sens, dlambda/dp = -<Y, dL/dp X> / <Y, M X>, for
 * p = Re, alpha, beta.
 * x, psi (device, [n_pencils][3N] complex): initial right and left iterates on entry (nonzero
 * components along the wanted eigenvectors), the normalised right and left prognostic
 * eigenvectors on exit.  out (device, [n_pencils][10] doubles): lambda (re, im),
 * dlambda/dRe, dlambda/dalpha, dlambda/dbeta (re, im each), and the relative residuals
 * |Phi x - mu x| / |Phi x| and |Phi^H psi - conj(mu) psi| / |Phi^H psi| of the last iterates
 * (mu = psi^H Phi x / psi^H x), which tell whether the iteration converged.
 * 1 <= n_pencils <= batch; SPADJ_ERR_INVALID for a singular shifted pencil (sigma on an
 * eigenvalue) or Re <= 0.  Synchronises the problem's stream before returning. */
spadj_status spadj_eigen(spadj_problem* prob, int n_pencils, const double* pencil_params, const double* shifts,
                         int n_iter, double* x, double* psi, double* out);

/* One-line description of the last failure on this problem (or of the last failed
 * spadj_create when prob is NULL).  Never NULL. */
const char* spadj_last_error(const spadj_problem* prob);

#ifdef __cplusplus
}
#endif

#endif /* SPADJ_H */
