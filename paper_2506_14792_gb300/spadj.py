"""ctypes binding of the C-ABI in include/spadj.h (argument marshalling only).

Every function of the header is exposed under the same name and takes raw device
pointers, as the C-ABI does; ``Problem`` is a small convenience wrapper that takes
torch CUDA tensors (float64 or complex128), checks their sizes and passes their
pointers.  All arithmetic runs in the CUDA kernels of libspadj.so.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libspadj.so")

SPADJ_OK = 0
SPADJ_ERR_INVALID = -1
SPADJ_ERR_NOMEM = -2
SPADJ_ERR_CUDA = -3
SPADJ_ERR_NONFINITE = -4
SPADJ_ERR_TIMEOUT = -5
SPADJ_ERR_UNSUPPORTED = -6

SPADJ_BURGERS1D = 0
SPADJ_RB2D = 1
SPADJ_KOLMOGOROV2D = 2
SPADJ_COUETTE3D = 3
SPADJ_SHEAR_EVP = 4

SPADJ_SBDF1 = 1
SPADJ_SBDF2 = 2
SPADJ_RK222 = 3
SPADJ_SBDF3 = 4
SPADJ_SBDF4 = 5
SPADJ_RK443 = 6

SPADJ_OBJ_ENERGY = 0
SPADJ_OBJ_FOURDVAR = 1
SPADJ_OBJ_GAIN = 2
SPADJ_OBJ_ENERGY_INTEGRAL = 3

C2G, G2C, C2G_ADJ, G2C_ADJ = 0, 1, 2, 3


class SpadjError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("spadj status %d: %s" % (status, msg))
        self.status = status


class spadj_desc(ctypes.Structure):
    _fields_ = [("eq", ctypes.c_int), ("scheme", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("length", ctypes.c_double * 3), ("params", ctypes.c_double * 4), ("dt", ctypes.c_double),
                ("batch", ctypes.c_int), ("nonlinear", ctypes.c_int), ("batch_n", ctypes.POINTER(ctypes.c_int)),
                ("closure", ctypes.c_int)]


_lib = None
_vp = ctypes.c_void_p
_SIGS = {
    "spadj_create": (ctypes.c_int, [ctypes.POINTER(spadj_desc), _vp, ctypes.POINTER(_vp)]),
    "spadj_destroy": (ctypes.c_int, [_vp]),
    "spadj_state_len": (ctypes.c_size_t, [_vp, ctypes.c_int]),
    "spadj_transform": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "spadj_transform_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "spadj_eval_F": (ctypes.c_int, [_vp, _vp, _vp]),
    "spadj_eval_F_jvp": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "spadj_eval_F_vjp": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "spadj_solve": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "spadj_vjp": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]),
    "spadj_resolvent": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int, _vp, _vp]),
    "spadj_hvp": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "spadj_checkpoint_schedule_host": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int,
                                                      ctypes.POINTER(ctypes.c_int)]),
    "spadj_set_dt_schedule": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "spadj_eigen": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, _vp, _vp]),
    "spadj_set_observations": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int]),
    "spadj_set_option": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "spadj_autotune": (ctypes.c_int, [_vp]),
    "spadj_set_params": (ctypes.c_int, [_vp, _vp]),
    "spadj_restrict": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "spadj_closure_conv": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "spadj_couette_pencil_solve_host": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                        ctypes.c_double, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "spadj_adam": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, _vp, _vp, _vp]),
    "spadj_checkpoint_schedule": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "spadj_forward": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "spadj_tangent": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "spadj_adjoint": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, _vp]),
    "spadj_step_forward": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "spadj_step_tangent": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "spadj_step_adjoint": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]),
    "spadj_objective": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, _vp]),
    "spadj_gradient": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp, _vp]),
    "spadj_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
    "spadj_timing_report": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_long)]),
    "spadj_last_error": (ctypes.c_char_p, [_vp]),
    "spadj_fp64_peak": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]),
}


def fp64_peak(stream=None, iters=200000):
    """Measured FP64 FMA throughput of the current device (GFLOP/s, timed duration in ms)."""
    import torch
    st = torch.cuda.current_stream() if stream is None else stream
    g, ms = ctypes.c_double(), ctypes.c_double()
    _chk(None, lib().spadj_fp64_peak(ctypes.c_void_p(st.cuda_stream), int(iters), ctypes.byref(g), ctypes.byref(ms)))
    return g.value, ms.value


def lib():
    """Load libspadj.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libspadj.so is not built (run paper_2506_14792_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _chk(handle, st):
    if st != SPADJ_OK:
        raise SpadjError(st, lib().spadj_last_error(handle).decode())


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _as_f64(t, n, name):
    import torch
    if t.is_complex():
        t = torch.view_as_real(t)
    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("%s must be a contiguous float64/complex128 CUDA tensor" % name)
    if n is not None and t.numel() != n:
        raise ValueError("%s has %d float64 elements, expected %d" % (name, t.numel(), n))
    return t


def checkpoint_schedule(n_steps, slots, host_slots=0):
    """Host-side binomial checkpoint schedule: list of (type, a, b, slot) actions; with
    host_slots > 0 the two-level (device + host) schedule."""
    n = ctypes.c_int()
    if host_slots:
        call = lambda buf, m: lib().spadj_checkpoint_schedule_host(n_steps, slots, host_slots, buf, m, ctypes.byref(n))
    else:
        call = lambda buf, m: lib().spadj_checkpoint_schedule(n_steps, slots, buf, m, ctypes.byref(n))
    _chk(None, call(None, 0))
    buf = (ctypes.c_int * (4 * n.value))()
    _chk(None, call(buf, n.value))
    return [tuple(buf[4 * i:4 * i + 4]) for i in range(n.value)]


def couette_pencil_solve_host(n_z, alpha, beta, re, a0, v, transpose=False, base=0):
    """Host banded step solve of one plane-Couette pencil (test support; no GPU): v is a numpy
    complex array of 3 n_z values (u, v, w blocks); returns the solution (or the adjoint map's
    result) as a new numpy array."""
    import numpy as np
    src = np.ascontiguousarray(v, dtype=np.complex128)
    if src.size != 3 * n_z:
        raise ValueError("couette_pencil_solve_host: v must hold 3 n_z complex values")
    out = np.zeros_like(src)
    _chk(None, lib().spadj_couette_pencil_solve_host(int(n_z), float(alpha), float(beta), float(re), float(a0),
                                                      int(base), int(bool(transpose)),
                                                      src.ctypes.data_as(ctypes.c_void_p),
                                                      out.ctypes.data_as(ctypes.c_void_p)))
    return out


CK_ADVANCE, CK_STORE, CK_RESTORE, CK_ADJOINT, CK_FREE, CK_OBJECTIVE = range(6)


class Problem:
    """Owns one spadj_problem; methods take torch CUDA tensors."""

    def __init__(self, eq, scheme, n, length, params, dt, batch=1, nonlinear=True, stream=None, batch_n=None,
                 closure=False):
        import torch
        d = spadj_desc()
        d.eq, d.scheme = eq, scheme
        for i, v in enumerate(list(n)[:3]):
            d.n[i] = int(v)
        for i, v in enumerate(list(length)[:3]):
            d.length[i] = float(v)
        for i, v in enumerate(list(params)[:4]):
            d.params[i] = float(v)
        d.dt, d.batch, d.nonlinear = float(dt), int(batch), int(bool(nonlinear))
        d.closure = int(bool(closure))
        if batch_n is not None:
            self._batch_n = (ctypes.c_int * len(batch_n))(*[int(v) for v in batch_n])
            d.batch_n = ctypes.cast(self._batch_n, ctypes.POINTER(ctypes.c_int))
        self.desc = d
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        st = lib().spadj_create(ctypes.byref(d), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        _chk(None, st)
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().spadj_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def state_len(self, which=0):
        return int(lib().spadj_state_len(self.h, which))

    def transform(self, kind, inp, out):
        nin = self.state_len(3 if kind in (C2G, G2C_ADJ) else 1)
        nout = self.state_len(1 if kind in (C2G, G2C_ADJ) else 3)
        _chk(self.h, lib().spadj_transform(self.h, kind, _ptr(_as_f64(inp, nin, "in")), _ptr(_as_f64(out, nout, "out"))))
        return out

    def eval_F(self, x, f):
        n = self.state_len(0)
        _chk(self.h, lib().spadj_eval_F(self.h, _ptr(_as_f64(x, n, "x")), _ptr(_as_f64(f, n, "f"))))
        return f

    def eval_F_jvp(self, x, dx, df):
        n = self.state_len(0)
        _chk(self.h, lib().spadj_eval_F_jvp(self.h, _ptr(_as_f64(x, n, "x")), _ptr(_as_f64(dx, n, "dx")),
                                             _ptr(_as_f64(df, n, "df"))))
        return df

    def eval_F_vjp(self, x, y, out):
        n = self.state_len(0)
        _chk(self.h, lib().spadj_eval_F_vjp(self.h, _ptr(_as_f64(x, n, "x")), _ptr(_as_f64(y, n, "y")),
                                             _ptr(_as_f64(out, n, "out"))))
        return out

    def solve(self, v, x, transpose=False):
        n = self.state_len(0)
        _chk(self.h, lib().spadj_solve(self.h, int(bool(transpose)), _ptr(_as_f64(v, n, "v")), _ptr(_as_f64(x, n, "x"))))
        return x

    def forward(self, n_steps, x0, x_out, traj=None):
        n = self.state_len(0)
        tp = None if traj is None else _ptr(_as_f64(traj, n * (n_steps + 1), "traj"))
        _chk(self.h, lib().spadj_forward(self.h, n_steps, _ptr(_as_f64(x0, n, "x0")), _ptr(_as_f64(x_out, n, "x_out")), tp))
        return x_out

    def tangent(self, n_steps, x0, dx0, dx_out):
        n = self.state_len(0)
        _chk(self.h, lib().spadj_tangent(self.h, n_steps, _ptr(_as_f64(x0, n, "x0")), _ptr(_as_f64(dx0, n, "dx0")),
                                          _ptr(_as_f64(dx_out, n, "dx_out"))))
        return dx_out

    def adjoint(self, n_steps, traj, y_final, grad_x0, grad_p=None):
        n = self.state_len(0)
        gp = None if grad_p is None else _ptr(_as_f64(grad_p, self.state_len(2), "grad_p"))
        _chk(self.h, lib().spadj_adjoint(self.h, n_steps, _ptr(_as_f64(traj, n * (n_steps + 1), "traj")),
                                          _ptr(_as_f64(y_final, n, "y_final")), _ptr(_as_f64(grad_x0, n, "grad_x0")),
                                          gp))
        return grad_x0

    def step_forward(self, n, s_n, s_np1):
        """Restart state s_{n+1} from s_n (spadj_state_len(4) float64 each)."""
        m = self.state_len(4)
        _chk(self.h, lib().spadj_step_forward(self.h, int(n), _ptr(_as_f64(s_n, m, "s_n")),
                                               _ptr(_as_f64(s_np1, m, "s_np1"))))
        return s_np1

    def step_tangent(self, n, s_n, ds_n, ds_np1):
        m = self.state_len(4)
        _chk(self.h, lib().spadj_step_tangent(self.h, int(n), _ptr(_as_f64(s_n, m, "s_n")),
                                               _ptr(_as_f64(ds_n, m, "ds_n")), _ptr(_as_f64(ds_np1, m, "ds_np1"))))
        return ds_np1

    def step_adjoint(self, n, x_n, y_np1, y_n, src=None, gp_accum=None):
        """Adjoint state y_n from y_{n+1} (None = zero) at the primal state x_n; src = dJ/dX_n."""
        n0, m = self.state_len(0), self.state_len(5)
        yp = None if y_np1 is None else _ptr(_as_f64(y_np1, m, "y_np1"))
        sp = None if src is None else _ptr(_as_f64(src, n0, "src"))
        gp = None if gp_accum is None else _ptr(_as_f64(gp_accum, self.state_len(2), "gp_accum"))
        _chk(self.h, lib().spadj_step_adjoint(self.h, int(n), _ptr(_as_f64(x_n, n0, "x_n")), yp, sp,
                                               _ptr(_as_f64(y_n, m, "y_n")), gp))
        return y_n

    def objective(self, x, J_dev, seed, objective=SPADJ_OBJ_ENERGY, obj_data=None):
        n = self.state_len(0)
        _chk(self.h, lib().spadj_objective(self.h, objective, _ptr(obj_data), _ptr(_as_f64(x, n, "x")),
                                            _ptr(_as_f64(J_dev, self.desc.batch, "J_dev")),
                                            _ptr(_as_f64(seed, n, "seed"))))
        return J_dev

    def gradient(self, x0, n_steps, grad_x0, objective=SPADJ_OBJ_ENERGY, obj_data=None, ckpt_slots=0,
                 grad_p=None, want_J=True):
        """Fills grad_x0; returns J per batch member (numpy, host) or None when want_J is False
        (then the call stays asynchronous on the stream)."""
        n = self.state_len(0)
        J = np.zeros(self.desc.batch, dtype=np.float64) if want_J else None
        jp = J.ctypes.data_as(ctypes.c_void_p) if want_J else None
        gp = None if grad_p is None else _ptr(_as_f64(grad_p, self.state_len(2), "grad_p"))
        _chk(self.h, lib().spadj_gradient(self.h, _ptr(_as_f64(x0, n, "x0")), n_steps, objective,
                                           _ptr(obj_data), ckpt_slots, jp,
                                           _ptr(_as_f64(grad_x0, n, "grad_x0")), gp))
        return J

    def set_observations(self, obs_steps, obs, kmax):
        n = self.state_len(0)
        steps = (ctypes.c_int * len(obs_steps))(*[int(v) for v in obs_steps])
        _chk(self.h, lib().spadj_set_observations(self.h, len(obs_steps), steps,
                                                   _ptr(_as_f64(obs, n * len(obs_steps), "obs")), int(kmax)))

    def set_params(self, params):
        _chk(self.h, lib().spadj_set_params(self.h, _ptr(_as_f64(params, self.state_len(2), "params"))))

    def restrict(self, n_fine, fine, coarse):
        """Spectral truncation of fine members (n_fine modes) to this problem's resolution."""
        B, Nc = self.desc.batch, self.desc.n[0]
        _chk(self.h, lib().spadj_restrict(self.h, int(n_fine), _ptr(_as_f64(fine, B * n_fine * n_fine, "fine")),
                                           _ptr(_as_f64(coarse, self.state_len(0), "coarse"))))
        return coarse

    def closure_conv(self, layer, mode, inp, out):
        """One 32 -> 32 closure convolution (mode 0 pre-activation, 1 input gradient); inp: int16/bfloat16
        CUDA tensor [pixels][32], out: float32 CUDA tensor of the same shape."""
        import torch
        if inp.dtype not in (torch.int16, torch.bfloat16) or out.dtype != torch.float32 or inp.numel() != out.numel():
            raise ValueError("closure_conv: bfloat16/int16 input and float32 output of equal size")
        if not (inp.is_cuda and out.is_cuda and inp.is_contiguous() and out.is_contiguous()):
            raise ValueError("closure_conv: contiguous CUDA tensors")
        _chk(self.h, lib().spadj_closure_conv(self.h, int(layer), int(mode), _ptr(inp), _ptr(out)))
        return out

    def adam(self, grad_p, t, m, v, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        """One Adam step on the closure parameters (m, v: caller-owned moments)."""
        n = self.state_len(2)
        _chk(self.h, lib().spadj_adam(self.h, _ptr(_as_f64(grad_p, n, "grad_p")), int(t), float(lr), float(b1),
                                       float(b2), float(eps), _ptr(_as_f64(m, n, "m")), _ptr(_as_f64(v, n, "v")),
                                       _ptr(_as_f64(params, n, "params"))))
        return params

    def set_option(self, option, value):
        _chk(self.h, lib().spadj_set_option(self.h, int(option), int(value)))

    def autotune(self):
        _chk(self.h, lib().spadj_autotune(self.h))

    def vjp(self, x0, n_steps, seed_steps, seeds, grad_x0, ckpt_slots=0):
        """grad_x0 = sum_i (dX_{seed_steps[i]}/dX_0)^T seeds[i]; seeds is [n_seeds][state] on the device."""
        n = self.state_len(0)
        steps = (ctypes.c_int * len(seed_steps))(*[int(s) for s in seed_steps])
        _chk(self.h, lib().spadj_vjp(self.h, _ptr(_as_f64(x0, n, "x0")), n_steps, ckpt_slots, len(seed_steps),
                                      steps, _ptr(_as_f64(seeds, n * len(seed_steps), "seeds")),
                                      _ptr(_as_f64(grad_x0, n, "grad_x0"))))
        return grad_x0

    def hvp(self, x0, v, n_steps, hv):
        """hv = Hessian of J = E(X_N) with respect to X_0 applied to v (tangent over adjoint)."""
        n = self.state_len(0)
        _chk(self.h, lib().spadj_hvp(self.h, _ptr(_as_f64(x0, n, "x0")), _ptr(_as_f64(v, n, "v")), int(n_steps),
                                      _ptr(_as_f64(hv, n, "hv"))))
        return hv

    def set_dt_schedule(self, dts):
        """Per-step sizes for later sweeps (SPADJ_RB2D); an empty sequence restores the constant dt."""
        import numpy as np
        d = np.ascontiguousarray(np.asarray(dts, dtype=np.float64).reshape(-1))
        _chk(self.h, lib().spadj_set_dt_schedule(self.h, int(d.size), d.ctypes.data_as(ctypes.c_void_p)))

    def eigen(self, pencil_params, shifts, n_iter, x, psi, out):
        """Leading eigenvalue nearest each shift and its sensitivities (SPADJ_SHEAR_EVP).
        pencil_params: host sequence of (alpha, beta, Re); shifts: host sequence of complex
        shifts; x, psi: [P][3N] complex128 CUDA iterates (in) / eigenvectors (out); out:
        [P][10] float64 CUDA (lambda, dlambda/dRe, dlambda/dalpha, dlambda/dbeta, residuals)."""
        import numpy as np
        prm = np.ascontiguousarray(np.asarray(pencil_params, dtype=np.float64).reshape(-1, 3))
        P = prm.shape[0]
        sh = np.asarray(shifts, dtype=np.complex128).reshape(P)
        shv = np.ascontiguousarray(np.stack([sh.real, sh.imag], axis=1))
        H = 3 * self.desc.n[2]
        _chk(self.h, lib().spadj_eigen(self.h, P, prm.ctypes.data_as(ctypes.c_void_p),
                                        shv.ctypes.data_as(ctypes.c_void_p), int(n_iter),
                                        _ptr(_as_f64(x, 2 * P * H, "x")), _ptr(_as_f64(psi, 2 * P * H, "psi")),
                                        _ptr(_as_f64(out, 10 * P, "out"))))
        return out

    def resolvent(self, omega, n_iter, f, gains):
        """Leading energy-norm resolvent gain per (kx, ky) pencil at frequency omega (power
        iteration); f: initial forcing in, leading forcing out; gains: [Ny][Nx/2] float64."""
        n = self.state_len(0)
        _chk(self.h, lib().spadj_resolvent(self.h, float(omega), int(n_iter), _ptr(_as_f64(f, n, "f")),
                                            _ptr(_as_f64(gains, self.desc.n[1] * (self.desc.n[0] // 2), "gains"))))
        return gains

    KERNEL_CLASSES = ("z_transform", "x_fft", "pointwise", "pencil_solve", "objective", "fused_trajectory", "y_fft",
                      "gram", "cnn")

    def timing(self, enable=True):
        _chk(self.h, lib().spadj_timing(self.h, int(bool(enable))))

    def timing_report(self):
        """{class: (ms, flops, launches)} since timing was enabled."""
        out = {}
        for k, name in enumerate(self.KERNEL_CLASSES):
            ms, fl, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_long()
            _chk(self.h, lib().spadj_timing_report(self.h, k, ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(n)))
            if n.value:
                out[name] = (ms.value, fl.value, n.value)
        return out
