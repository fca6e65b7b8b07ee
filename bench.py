"""Benchmark: forward+adjoint gradient evaluations in dof*steps/s.

One bench "step" is one whole gradient evaluation of the workload (forward sweep with
checkpoint/trajectory writes, objective, adjoint sweep) over one batch of synthetic
input resident in HBM.  The GPU arm runs the CUDA library through its C-ABI; the
reference arm (``--impl reference``) times the FP64 CPU oracle on a bounded sample of
the same workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                       [--workload rb|burgers|kolmogorov|couette|poiseuille_evp|couette_resolvent]
                       [--scheme rk443|sbdf1..sbdf4] [--op integral|hvp] [--dt-blocks B] [--omega W]
Under torchrun (N > 1) each rank runs an independent replica / shard; the time is the
max over ranks and the value counts the units of all ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import time

# the CPU oracle baseline is reported per core: keep numpy's BLAS single-threaded
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Nominal FP64 peak, for context: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz (GB300 FP64 1.25 TFLOP/s).
# The roofline uses the peak measured on the run's own GPU (measure_fp64_peak).
FP64_NOMINAL_GFLOPS = 152 * 2 * 2 * 2.07


def measure_fp64_peak(gpu_index, iters=100000):
    """FP64 FMA throughput of this GPU from the library's probe kernel (independent FMA chains,
    occupancy-sized grid, CUDA events), best of three launches, with the SM clocks sampled while it
    runs."""
    from paper_2506_14792_gb300 import spadj
    clk = ClockSampler(gpu_index)
    clk.start()
    time.sleep(0.3)
    runs = [spadj.fp64_peak(iters=iters) for _ in range(3)]
    clocks = clk.stop()
    g, ms = max(runs)
    return {"gflops": g, "ms": ms, "runs_gflops": [r[0] for r in runs], "clocks": clocks,
            "how": "spadj_fp64_peak: 8 independent FMA chains per thread, %d FMAs each, occupancy-sized grid, "
                   "best of 3" % iters}


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of the GB300s (GB/s), or the recipe's fallback."""
    try:
        with open(PEAKS_PATH) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def bf16_peak_gflops():
    """Measured dense BF16 tensor rate (burst, GFLOP/s) and its source, or the recipe's fallback."""
    try:
        with open(PEAKS_PATH) as f:
            return 1e3 * float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, ValueError, KeyError):
        return 1.9e6, "fallback"


def hbm_fraction(traffic, avg_launch_s):
    """DRAM bytes of one launch of the dominant kernel over its CUDA-event duration, against the
    measured HBM roof (the metric's "% HBM roofline"); None without an ncu traffic figure."""
    if not traffic:
        return None
    peak, src = hbm_peak_gbs()
    achieved = traffic / avg_launch_s / 1e9
    return {"achieved_gbs": achieved, "peak_gbs": peak, "frac": achieved / peak, "peak_source": src}


# DRAM traffic (bytes per launch) of the dominant kernel from an ncu capture, keyed by
# (workload, kernel class); None until measured for the current kernels.
TRAFFIC = {
    # cou_solve_kernel: 81.66 MB read + 1.44 MB written per launch on the 64x32x32 capture (equal to
    # the algorithmic operator + vector bytes); scaled to 128x64x64 by the operator bytes (16x) and
    # the vector bytes (8x), averaged over the forward (5 vectors) and transposed (2) launches
    ("couette3d_128x64x64_Re1000_sbdf2_4000steps_gain", "pencil_solve"): 1.252e9,
    # xfft_kernel, one row per CTA (the setting the problem picks): dram read + write per launch on
    # the RB capture (8-job 1.23 MB, 6-job 2.41 MB, 3-job 0.64 / 2.41 MB), weighted by the launch mix
    # of the gradient (484 : 200 : 200 : 380); the working set is L2-resident, so this is the
    # cold-cache fill ncu sees after its cache flush
    ("rayleigh_benard2d_256x64_Ra1e6_rk222_2000steps", "x_fft"): 1.68e6,
    # evp_iter_kernel, full bench launch (608 pencils, 100 iterations): 32.07 GB read + 7.4 MB
    # written, against 35.9 GB of operator rows streamed by the algorithm (the rest hits in L2)
    ("poiseuille_evp_N64_608pencils_Re8000_100iter", "pencil_solve"): 3.2075e10,
    # Burgers trajectory + adjoint kernels, captured at 50 steps (forward: 36 MB read + 1.650 GB of
    # trajectory written; adjoint: 1.715 GB of trajectory read + 44 MB written), trajectory bytes
    # scaled to 1000 steps by (1001 / 51), averaged over the two launches of a gradient
    ("burgers1d_N256_sbdf2_1000steps", "fused_trajectory"): 3.31e10,
    # kol_persistent: no capture of the gradient's own sweeps yet (the captured launches were the
    # 5-step forward sweeps that generate the observations: 6.76 GB read + 4.88 GB written each,
    # about 2.3 GB per step of the 64 members' mixed-space arrays)
    ("kolmogorov2d_batch64_mixed128-512_Re100_sbdf2_2000steps_4dvar8", "fused_trajectory"): None,
}


# kernels whose per-launch traffic is their stored trajectory: (steps the TRAFFIC figure is quoted
# at, stored states as a function of the workload); other entries are per launch and independent
# of the horizon
TRAFFIC_STEPS = {
    ("burgers1d_N256_sbdf2_1000steps", "fused_trajectory"): (1001, lambda wl: wl.nsteps + 1),
}


def traffic_for(wl, dom):
    """DRAM bytes per launch of the dominant kernel at this workload's horizon (None if never
    captured)."""
    t = TRAFFIC.get((wl.name, dom))
    sc = TRAFFIC_STEPS.get((wl.name, dom))
    if t is not None and sc is not None:
        t = t * sc[1](wl) / sc[0]
    return t


def fp64_flops_real_fft(M):
    """Conventional flop count of one real FFT of length M (half of 5 M log2 M)."""
    return 2.5 * M * np.log2(M)


# ---------------------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------------------

class Burgers:
    """1D viscous Burgers, N=256, nu=0.01, SBDF2 dt=1e-3, 1000 steps, 16384 members."""
    name = "burgers1d_N256_sbdf2_1000steps"

    ORDERS = {"sbdf1": 1, "sbdf2": 2, "sbdf3": 3, "sbdf4": 4}

    def __init__(self, batch=16384, N=256, nsteps=1000, dt=1e-3, nu=0.01, seed=1, scheme="sbdf2", slots=0):
        self.B, self.N, self.nsteps, self.dt, self.nu, self.seed = batch, N, nsteps, dt, nu, seed
        self.dof = N
        self.K, self.M = N // 2, 3 * N // 2
        self.scheme = scheme
        self.slots = slots
        if scheme != "sbdf2" or batch != 16384 or slots:
            self.name = "burgers1d_N%d_%s_%dsteps%s%s" % (N, scheme, nsteps, "" if batch == 16384 else "_b%d" % batch,
                                                          "_ckpt%d" % slots if slots else "")

    def config(self):
        return {"workload": self.name, "N": self.N, "nu": self.nu, "dt": self.dt, "steps": self.nsteps,
                "batch": self.B, "scheme": self.scheme.upper(), "objective": "0.5||u(T)||^2",
                "checkpointing": ("binomial, %d restart-state slots" % self.slots) if self.slots else "store-all",
                "l2": "working set > L2 (%s %.1f GB)" % (
                    ("checkpoint slots", self.slots * self.ckpt_state_bytes()) if self.slots
                    else ("stored trajectory", self.traj_bytes() / 1e9))}

    def ckpt_state_bytes(self):
        """GB of one restart state (the (2s - 1) state blocks of an order-s SBDF step)."""
        return (2 * self.ORDERS[self.scheme] - 1) * self.B * self.K * 16 / 1e9

    def traj_bytes(self):
        return (self.nsteps + 1) * self.B * self.K * 16

    def units_per_step(self):
        return self.B * self.dof * self.nsteps


    def setup(self, device):
        import torch
        from paper_2506_14792_gb300 import spadj
        self.torch = torch
        self.sp = spadj
        sch = {"sbdf1": spadj.SPADJ_SBDF1, "sbdf2": spadj.SPADJ_SBDF2, "sbdf3": spadj.SPADJ_SBDF3,
               "sbdf4": spadj.SPADJ_SBDF4}[self.scheme]
        self.p = spadj.Problem(spadj.SPADJ_BURGERS1D, sch, [self.N], [2 * np.pi], [self.nu], self.dt, batch=self.B)
        self.X0_host = synthetic.burgers_ic(self.N, batch=self.B, seed=self.seed)
        self.x0 = torch.from_numpy(self.X0_host).to(device)
        if self.slots:
            self.traj = None
            self.xN = torch.empty((self.B, self.K), dtype=torch.complex128, device=device)
        else:
            self.traj = torch.empty((self.nsteps + 1, self.B, self.K), dtype=torch.complex128, device=device)
            self.xN = self.traj[-1]
        self.J = torch.empty(self.B, dtype=torch.float64, device=device)
        self.seedv = torch.empty((self.B, self.K), dtype=torch.complex128, device=device)
        self.grad = torch.empty((self.B, self.K), dtype=torch.complex128, device=device)
        self.x0_pin = torch.from_numpy(self.X0_host).pin_memory()
        self.grad_pin = torch.empty((self.B, self.K), dtype=torch.complex128).pin_memory()
        self.x0_dev2 = torch.empty_like(self.x0)


    flush_l2 = False

    def step(self, ev=None):
        """Device-resident step: forward (trajectory stored), objective, adjoint sweep; with
        checkpoint slots the library's checkpointed gradient (forward to the slots, reverse sweep
        with recomputation)."""
        if self.slots:
            self.p.gradient(self.x0, self.nsteps, self.grad, ckpt_slots=self.slots, want_J=False)
            return
        self.p.forward(self.nsteps, self.x0, self.xN, self.traj)
        self.p.objective(self.xN, self.J, self.seedv)
        self.p.adjoint(self.nsteps, self.traj, self.seedv, self.grad)

    def forward_step(self):
        self.p.forward(self.nsteps, self.x0, self.xN)

    def e2e_step(self):
        """Public API call with host buffers: pinned H2D of x0, spadj_gradient (J to host), D2H of grad."""
        self.x0_dev2.copy_(self.x0_pin, non_blocking=True)
        J = self.p.gradient(self.x0_dev2, self.nsteps, self.grad, ckpt_slots=self.slots)
        self.grad_pin.copy_(self.grad, non_blocking=True)
        return J

    def e2e_bytes(self):
        return self.B * self.K * 16, self.B * self.K * 16 + self.B * 8

    # CPU oracle on a bounded sample
    def cpu_sample(self):
        from oracle import burgers as ob
        o = ob.Burgers(self.N, self.nu)
        Bs = min(256, self.B)
        X0 = self.X0_host[:Bs] if hasattr(self, "X0_host") else synthetic.burgers_ic(self.N, batch=Bs, seed=self.seed)
        t = time.perf_counter()
        ob.gradient(o, X0, self.nsteps, self.dt, order=self.ORDERS[self.scheme])
        el = time.perf_counter() - t
        return Bs * self.dof * self.nsteps / el, "%d members x %d steps (gradient, numpy FP64)" % (Bs, self.nsteps), el


class RayleighBenard:
    """2D Rayleigh-Benard, Fourier(x) 256 x Chebyshev(z) 64 tau, Ra=1e6, Pr=1, no-slip,
    RK222 dt=1e-3, 2000 steps, kinetic energy at T, binomial checkpointing (64 slots)."""
    name = "rayleigh_benard2d_256x64_Ra1e6_rk222_2000steps"

    def __init__(self, Nx=256, Nz=64, Ra=1e6, Pr=1.0, dt=1e-3, nsteps=2000, slots=64, seed=2, amp=1e-3,
                 scheme="rk222", dt_blocks=0):
        self.Nx, self.Nz, self.Ra, self.Pr, self.dt, self.nsteps = Nx, Nz, Ra, Pr, dt, nsteps
        self.slots, self.seed, self.amp = slots, seed, amp
        self.dof = 3 * Nx * Nz
        self.B = 1
        self.flush_l2 = True
        self.scheme = scheme
        # dt_blocks > 0: step-size schedule alternating dt and dt/2 every dt_blocks steps (two
        # stage-operator sets, each factorised once and kept)
        self.dt_blocks = dt_blocks
        self.name = "rayleigh_benard2d_%dx%d_Ra1e6_%s_%dsteps%s" % (
            Nx, Nz, scheme, nsteps, "_dtblocks%d" % dt_blocks if dt_blocks else "")

    def schedule(self):
        return [self.dt * (0.5 if (n // self.dt_blocks) % 2 else 1.0) for n in range(self.nsteps)]

    def config(self):
        return {"workload": self.name, "Nx": self.Nx, "Nz": self.Nz, "Ra": self.Ra, "Pr": self.Pr, "dt": self.dt,
                "steps": self.nsteps, "scheme": {"rk222": "RK222 (ARS222)", "rk443": "RK443 (ARS443)"}[self.scheme],
                "objective": "kinetic energy at T",
                **({"dt_schedule": "dt and dt/2 alternating every %d steps" % self.dt_blocks}
                   if self.dt_blocks else {}),
                "checkpoint_slots": self.slots, "dof": self.dof,
                **({"parity": "J and dJ/dX_0 of this exact input and horizon match the FP64 oracle element by "
                              "element to 1e-10 relative (tests/test_gpu_rb.py::"
                              "test_full_horizon_gradient_matches_oracle_golden; the oracle's own rounding-order "
                              "spread at 2000 steps is 1.1e-14)"}
                   if (self.Nx, self.Nz, self.nsteps, self.scheme, self.dt_blocks) == (256, 64, 2000, "rk222", 0)
                   else {}),
                "l2": "L2 flushed between timed iterations (256 MB write); working set ~60 MB fits L2"}

    def units_per_step(self):
        return self.dof * self.nsteps

    def setup(self, device):
        import torch
        from paper_2506_14792_gb300 import spadj
        self.torch = torch
        sch = {"rk222": spadj.SPADJ_RK222, "rk443": spadj.SPADJ_RK443}[self.scheme]
        self.p = spadj.Problem(spadj.SPADJ_RB2D, sch, [self.Nx, self.Nz], [4.0], [self.Ra, self.Pr], self.dt)
        if self.dt_blocks:
            self.p.set_dt_schedule(self.schedule())
        self.s0 = synthetic.rb_ic(self.Nx, self.Nz, seed=self.seed, amp=self.amp)
        shape = (3, self.Nx // 2, self.Nz)
        self.x0 = torch.from_numpy(self.s0).to(device)
        self.grad = torch.empty(shape, dtype=torch.complex128, device=device)
        self.x0_pin = torch.from_numpy(self.s0).pin_memory()
        self.grad_pin = torch.empty(shape, dtype=torch.complex128).pin_memory()
        self.x0_dev2 = torch.empty_like(self.x0)
        self.launches = None

    def step(self, ev=None):
        self.p.gradient(self.x0, self.nsteps, self.grad, ckpt_slots=self.slots, want_J=False)

    def forward_step(self):
        self.p.forward(self.nsteps, self.x0, self.x0_dev2)

    def e2e_step(self):
        self.x0_dev2.copy_(self.x0_pin, non_blocking=True)
        J = self.p.gradient(self.x0_dev2, self.nsteps, self.grad, ckpt_slots=self.slots)
        self.grad_pin.copy_(self.grad, non_blocking=True)
        return J

    def e2e_bytes(self):
        n = self.s0.nbytes
        return n, n + 8

    def cpu_sample(self, nsteps=6):
        """Oracle gradient (store-all) over the first `nsteps` steps of the same workload."""
        from oracle import imex
        from oracle import rayleigh_benard as orb
        tab = imex.rk443_tableaux() if self.scheme == "rk443" else None
        if not hasattr(self, "_oracle"):
            self._oracle = orb.RayleighBenard(self.Nx, self.Nz, self.Ra, self.Pr)
            orb.gradient(self._oracle, self._oracle.pencils(synthetic.rb_ic(self.Nx, self.Nz, seed=self.seed,
                                                                                amp=self.amp)), 1, self.dt, tab)
        o = self._oracle
        X0 = o.pencils(synthetic.rb_ic(self.Nx, self.Nz, seed=self.seed, amp=self.amp))
        dt = self.schedule()[:nsteps] if self.dt_blocks else self.dt
        t = time.perf_counter()
        orb.gradient(o, X0, nsteps, dt, tab)
        el = time.perf_counter() - t
        return (self.dof * nsteps / el,
                "%d of %d steps of the same gradient (forward+adjoint, store-all, numpy/scipy FP64, "
                "factorisations cached)" % (nsteps, self.nsteps), el)


class KolmogorovBatch:
    """Batched 2D Kolmogorov, Re=100, forcing sin(4y), 64 members (16 each at 128^2, 256^2,
    384^2, 512^2) in one persistent launch per sweep, SBDF2 dt=5e-4, 2000 steps, 4D-Var misfit
    to 8 observation times (every 250 steps, |k| <= 32).  Observations come from a separate
    truth run of the same solver (synthetic data)."""
    name = "kolmogorov2d_batch64_mixed128-512_Re100_sbdf2_2000steps_4dvar8"

    def __init__(self, nsteps=2000, dt=5e-4, Re=100.0, slots=0):
        self.slots = slots
        if slots:
            self.name = self.name + "_seg%d" % slots
        self.res = [128, 256, 384, 512]
        self.sizes = [self.res[i // 16] for i in range(64)]
        self.nsteps, self.dt, self.Re = nsteps, dt, Re
        self.dof = sum(n * n for n in self.sizes)
        self.flush_l2 = False
        self.B = 64

    def config(self):
        return {"workload": self.name, "members": 64, "resolutions": self.res, "Re": self.Re, "dt": self.dt,
                "steps": self.nsteps, "observations": self.obs_steps(), "dof_per_step": self.dof,
                "checkpointing": ("%d segments (restart state at each segment start, one segment recomputed "
                                  "per reverse launch)" % self.slots) if self.slots else "store-all",
                "l2": "working set > L2 (%s %.0f GB)" % (
                    "segment buffer and restart states" if self.slots else "stored trajectory",
                    16 * sum((n // 2) * n for n in self.sizes) * (
                        (-(-self.nsteps // self.slots) + 1 + 3 * self.slots) if self.slots else (self.nsteps + 1)) / 1e9)}

    def obs_steps(self):
        k = max(1, self.nsteps // 8)
        return [k * (i + 1) for i in range(8)]

    def units_per_step(self):
        return self.dof * self.nsteps

    def setup(self, device):
        import torch
        from paper_2506_14792_gb300 import spadj
        self.torch = torch
        self.sp = spadj
        self.p = spadj.Problem(spadj.SPADJ_KOLMOGOROV2D, spadj.SPADJ_SBDF2, [128], [2 * np.pi], [self.Re, 0.0],
                               self.dt, batch=64, batch_n=self.sizes)
        pack = lambda arrs: np.concatenate([a.ravel() for a in arrs])
        self.x0_host = pack([synthetic.kolmogorov_ic(n, 100 + i) for i, n in enumerate(self.sizes)])
        truth = torch.from_numpy(pack([synthetic.kolmogorov_ic(n, 5000 + i) for i, n in enumerate(self.sizes)])).to(device)
        # observations: truth states at the observation steps (segments of the same solver),
        # low-passed by the objective's observation operator inside the library
        obs, cur, last = [], truth, 0
        for k in self.obs_steps():
            nxt = torch.empty_like(cur)
            self.p.forward(k - last, cur, nxt)
            obs.append(nxt)
            cur, last = nxt, k
        self.p.set_observations(self.obs_steps(), torch.stack(obs).contiguous(), 32)
        self.p.autotune()
        self.x0 = torch.from_numpy(self.x0_host).to(device)
        self.grad = torch.empty_like(self.x0)
        self.x0_pin = torch.from_numpy(self.x0_host).pin_memory()
        self.grad_pin = torch.empty(self.x0.shape, dtype=torch.complex128).pin_memory()
        self.x0_dev2 = torch.empty_like(self.x0)

    def step(self, ev=None):
        self.p.gradient(self.x0, self.nsteps, self.grad, objective=self.sp.SPADJ_OBJ_FOURDVAR, ckpt_slots=self.slots,
                        want_J=False)

    def forward_step(self):
        self.p.forward(self.nsteps, self.x0, self.x0_dev2)

    def e2e_step(self):
        self.x0_dev2.copy_(self.x0_pin, non_blocking=True)
        J = self.p.gradient(self.x0_dev2, self.nsteps, self.grad, objective=self.sp.SPADJ_OBJ_FOURDVAR,
                            ckpt_slots=self.slots)
        self.grad_pin.copy_(self.grad, non_blocking=True)
        return J

    def e2e_bytes(self):
        n = self.x0_host.nbytes
        return n, n + 8 * 64

    def cpu_sample(self, nsteps=4):
        """Oracle 4D-Var gradient of one 128^2 and one 512^2 member over a short window, scaled to
        the batch's dof mix (dof*steps/s of the two members together)."""
        from oracle import kolmogorov as okol
        t = time.perf_counter()
        d = 0
        for n in (128, 512):
            o = okol.Kolmogorov(n, self.Re)
            X0 = o.project(synthetic.kolmogorov_ic(n, 7))
            mask = o.lowpass_mask(32)
            obs = np.stack([np.zeros_like(X0)] * 2)
            okol.fourdvar_gradient(o, X0, nsteps, self.dt, [nsteps // 2, nsteps], obs, mask)
            d += n * n
        el = time.perf_counter() - t
        return d * nsteps / el, "one 128^2 and one 512^2 member, %d-step 4D-Var gradient (numpy FP64)" % nsteps, el


class Couette:
    """3D plane Couette, Fourier(x, y) 128 x 64 x Chebyshev(z) 64 tau, Re=1000, SBDF2 dt=5e-3,
    4000 steps, energy gain E(T)/E(0) of a divergence-free initial field of norm 1e-4,
    checkpoint slots sized to a 180 GB HBM budget."""
    name = "couette3d_128x64x64_Re1000_sbdf2_4000steps_gain"

    def __init__(self, Nx=128, Ny=64, Nz=64, Re=1000.0, dt=5e-3, nsteps=4000, seed=5, norm=1e-4, budget=180e9,
                 op="gain"):
        self.Nx, self.Ny, self.Nz, self.Re, self.dt, self.nsteps = Nx, Ny, Nz, Re, dt, nsteps
        self.seed, self.norm, self.budget = seed, norm, budget
        self.dof = 3 * Nx * Ny * Nz
        self.B = 1
        self.flush_l2 = False
        self.slot_bytes = 3 * 16 * 3 * (Nx // 2) * Ny * Nz  # (x_n, x_{n-1}, f_{n-1})
        # op: "gain" (gradient of E(T)/E(0)), "integral" (gradient of the time integral of E,
        # carried as an extra equation) or "hvp" (Hessian of E(X_N) applied to a direction,
        # tangent over adjoint, trajectory and tangent stored)
        self.op = op
        if op != "gain":
            self.name = "couette3d_%dx%dx%d_Re1000_sbdf2_%dsteps_%s" % (Nx, Ny, Nz, nsteps, op)
            self.metric = {"integral": "forward+adjoint gradient of the time-integrated energy dof*steps/s at 1e-10 "
                                       "rel vs FP64 oracle",
                           "hvp": "Hessian-vector product (tangent over adjoint) dof*steps/s at 1e-10 rel vs FP64 "
                                  "oracle"}[op]

    @property
    def slots(self):
        return int(min(self.nsteps + 1, self.budget // self.slot_bytes))

    def config(self):
        return {"workload": self.name, "Nx": self.Nx, "Ny": self.Ny, "Nz": self.Nz, "Re": self.Re, "dt": self.dt,
                "steps": self.nsteps, "scheme": "SBDF1 -> SBDF2",
                "objective": {"gain": "energy gain E(T)/E(0)", "integral": "time integral of E (extra equation)",
                              "hvp": "E(X_N), Hessian-vector product"}[self.op],
                "checkpoint_slots": self.slots if self.op != "hvp" else "store-all (trajectory and tangent)",
                "dof": self.dof,
                "l2": "working set > L2 (pencil operators 4.8 GB read every step)"}

    def units_per_step(self):
        return self.dof * self.nsteps

    def _ic(self):
        u = synthetic.couette_ic(self.Nx, self.Ny, self.Nz, seed=self.seed, norm=self.norm)
        return np.ascontiguousarray(np.transpose(u, (0, 2, 1, 3)))  # library layout [3][Ny][Nx/2][Nz]

    def setup(self, device):
        import torch
        from paper_2506_14792_gb300 import spadj
        self.sp = spadj
        self.p = spadj.Problem(spadj.SPADJ_COUETTE3D, spadj.SPADJ_SBDF2, [self.Nx, self.Ny, self.Nz],
                               [4 * np.pi, 2 * np.pi], [self.Re], self.dt)
        self.s0 = self._ic()
        self.x0 = torch.from_numpy(self.s0).to(device)
        self.grad = torch.empty_like(self.x0)
        self.x0_pin = torch.from_numpy(self.s0).pin_memory()
        self.grad_pin = torch.empty(self.x0.shape, dtype=torch.complex128).pin_memory()
        self.x0_dev2 = torch.empty_like(self.x0)
        if self.op == "hvp":
            v = synthetic.couette_ic(self.Nx, self.Ny, self.Nz, seed=self.seed + 86, norm=self.norm)
            self.v = torch.from_numpy(np.ascontiguousarray(np.transpose(v, (0, 2, 1, 3)))).to(device)

    def _objective(self):
        return self.sp.SPADJ_OBJ_ENERGY_INTEGRAL if self.op == "integral" else self.sp.SPADJ_OBJ_GAIN

    def step(self, ev=None):
        if self.op == "hvp":
            self.p.hvp(self.x0, self.v, self.nsteps, self.grad)
            return
        self.p.gradient(self.x0, self.nsteps, self.grad, objective=self._objective(), ckpt_slots=self.slots,
                        want_J=False)

    def forward_step(self):
        self.p.forward(self.nsteps, self.x0, self.x0_dev2)

    def e2e_step(self):
        self.x0_dev2.copy_(self.x0_pin, non_blocking=True)
        if self.op == "hvp":
            self.p.hvp(self.x0_dev2, self.v, self.nsteps, self.grad)
            self.grad_pin.copy_(self.grad, non_blocking=True)
            return None
        J = self.p.gradient(self.x0_dev2, self.nsteps, self.grad, objective=self._objective(),
                            ckpt_slots=self.slots)
        self.grad_pin.copy_(self.grad, non_blocking=True)
        return J

    def e2e_bytes(self):
        n = self.s0.nbytes
        return n, n + 8

    def cpu_sample(self, nsteps=40, size=(32, 16, 32)):
        """Oracle gain gradient (store-all) on a reduced grid of the same equations: the dense
        per-pencil LU oracle cannot factor the 4096 full-size pencils within the sample budget."""
        from oracle import couette as oco
        from oracle import imex
        o = oco.Couette(*size, self.Re)
        X0 = o.pencils(synthetic.couette_ic(*size, seed=self.seed, norm=self.norm))
        oco.gain_gradient(o, X0, 1, self.dt)  # factorisations cached outside the timed sample
        t = time.perf_counter()
        if self.op == "integral":
            imex.integral_gradient(o, X0, nsteps, self.dt, o.energy, o.energy_grad)
        elif self.op == "hvp":
            X = imex.multistep_forward(o, X0, nsteps, self.dt)
            dX = imex.multistep_tangent(o, X, o.pencils(synthetic.couette_ic(*size, seed=self.seed + 86,
                                                                             norm=self.norm)), self.dt)
            imex.multistep_hvp(o, X, dX, lambda k: o.energy_grad(X[k]) if k == nsteps else None,
                               lambda k: o.energy_grad(dX[k]) if k == nsteps else None, self.dt)
        else:
            oco.gain_gradient(o, X0, nsteps, self.dt)
        el = time.perf_counter() - t
        dof = 3 * size[0] * size[1] * size[2]
        what = {"gain": "the gain gradient (forward+adjoint", "integral": "the time-integrated energy gradient "
                "(forward+adjoint", "hvp": "the Hessian-vector product (forward, tangent, adjoint and its tangent"}
        return (dof * nsteps / el,
                "reduced grid %dx%dx%d, %d steps of %s, store-all, numpy/scipy FP64, factorisations cached)"
                % (size + (nsteps, what[self.op])), el)


class PoiseuilleEvp:
    """Batched linear-stability eigenvalues of plane Poiseuille flow with their adjoint
    sensitivities (Parametric sensitivity example): 608 pencils (alpha 0.6..1.3 x beta 0..1.4,
    Re = 8000, N = 64 Chebyshev modes), shifts on the wall-mode branch lambda ~ -0.25 i alpha,
    100 shift-invert iterations per pencil (forward and adjoint together), then eigenvectors
    and dlambda/d(Re, alpha, beta).  One step = one spadj_eigen call."""
    name = "poiseuille_evp_N64_608pencils_Re8000_100iter"
    metric = "eigenvalue+sensitivity solves/s (leading mode, dlambda/d(Re, alpha, beta))"
    unit = "solves/s"

    def __init__(self, N=64, Re=8000.0, n_alpha=38, n_beta=16, n_iter=100, seed=12):
        self.N, self.Re, self.n_iter, self.seed = N, Re, n_iter, seed
        al = np.linspace(0.6, 1.3, n_alpha)
        be = np.linspace(0.0, 1.4, n_beta)
        self.cases = np.array([(a, b, Re) for b in be for a in al])
        self.P = len(self.cases)
        self.shifts = -0.25j * self.cases[:, 0]
        self.flush_l2 = False

    def config(self):
        return {"workload": self.name, "N": self.N, "Re": self.Re, "pencils": self.P, "iterations": self.n_iter,
                "base_flow": "plane Poiseuille U = 1 - z^2", "alpha": [0.6, 1.3], "beta": [0.0, 1.4],
                "l2": "pencil operators 359 MB > L2, re-read every iteration"}

    def units_per_step(self):
        return self.P

    def setup(self, device):
        import torch
        from paper_2506_14792_gb300 import stability
        self.p = stability.shear_evp_problem(self.N, "poiseuille", self.P)
        rng = np.random.default_rng(self.seed)
        H = 3 * self.N
        self.x_init = torch.tensor(rng.standard_normal((self.P, H)) + 1j * rng.standard_normal((self.P, H)))
        self.psi_init = torch.tensor(rng.standard_normal((self.P, H)) + 1j * rng.standard_normal((self.P, H)))
        self.x = self.x_init.to(device)
        self.psi = self.psi_init.to(device)
        self.out = torch.zeros((self.P, 10), dtype=torch.float64, device=device)
        self.out_host = torch.zeros((self.P, 10), dtype=torch.float64).pin_memory()

    def step(self):
        self.x.copy_(self.x_init, non_blocking=True)
        self.psi.copy_(self.psi_init, non_blocking=True)
        self.p.eigen(self.cases, self.shifts, self.n_iter, self.x, self.psi, self.out)
        self.out_host.copy_(self.out)

    def e2e_bytes(self):
        nv, H = 4 * self.N + 7, 3 * self.N
        h2d = self.P * (2 * nv * H * 16 + 2 * H * 16 + 5 * 8)  # operators T, RH; iterates; params, shifts
        return h2d, self.P * 10 * 8

    def cpu_sample(self, n=6):
        """Oracle: dense QZ eigenpairs with left vectors and eq. eigenvalue_sens for n pencils of
        the batch (numpy/scipy FP64)."""
        from oracle.shear_evp import ShearEVP
        e = ShearEVP(self.N, "poiseuille")
        idx = np.linspace(0, self.P - 1, n).astype(int)
        t = time.perf_counter()
        for i in idx:
            a, b, Re = self.cases[i]
            lam_all, X, Y = e.eigs(a, b, Re)
            j = int(np.argmin(np.abs(lam_all - self.shifts[i])))
            e.sensitivity(a, b, Re, lam_all[j], X[:, j], Y[:, j])
        el = time.perf_counter() - t
        return n / el, "%d of the %d pencils: dense QZ (left+right vectors) + sensitivities, N = %d" % (
            n, self.P, self.N), el


class CouetteResolvent:
    """Leading energy-norm resolvent gain of every (kx, ky) pencil of plane Couette flow at one
    frequency (the LBVP adjoint: the transposed pencil solves supply R^H), Re = 1000, by a batched
    power iteration on R^H G R f = sigma^2 G f.  One step = one spadj_resolvent call of n_iter
    iterations; the complex-shift pencil factorisations are built on the host at the first call
    for a frequency and kept (outside the timed region)."""
    metric = "resolvent gain power iterations (pencil*iterations/s, forward and adjoint pencil solves)"
    unit = "pencil*iterations/s"

    def __init__(self, Nx=64, Ny=32, Nz=32, Re=1000.0, omega=0.0, n_iter=50, seed=61):
        self.Nx, self.Ny, self.Nz, self.Re, self.omega, self.n_iter, self.seed = Nx, Ny, Nz, Re, omega, n_iter, seed
        self.P = (Nx // 2) * Ny
        self.name = "couette3d_%dx%dx%d_Re1000_resolvent_omega%g_%diter" % (Nx, Ny, Nz, omega, n_iter)
        self.flush_l2 = False

    def config(self):
        return {"workload": self.name, "Nx": self.Nx, "Ny": self.Ny, "Nz": self.Nz, "Re": self.Re,
                "omega": self.omega, "pencils": self.P, "iterations": self.n_iter,
                "l2": "pencil operators %.0f MB" % (2 * self.P * (3 * self.Nz) ** 2 * 16 / 1e6)}

    def units_per_step(self):
        return self.P * self.n_iter

    def setup(self, device):
        import torch
        from paper_2506_14792_gb300 import spadj
        self.p = spadj.Problem(spadj.SPADJ_COUETTE3D, spadj.SPADJ_SBDF2, [self.Nx, self.Ny, self.Nz],
                               [4 * np.pi, 2 * np.pi], [self.Re], 5e-3)
        shape = (3, self.Ny, self.Nx // 2, self.Nz)
        self.f_init = torch.from_numpy(synthetic.random_coeffs(shape, seed=self.seed))
        self.f = self.f_init.to(device)
        self.gains = torch.zeros((self.Ny, self.Nx // 2), dtype=torch.float64, device=device)
        self.gains_host = torch.zeros((self.Ny, self.Nx // 2), dtype=torch.float64).pin_memory()

    def step(self):
        self.f.copy_(self.f_init, non_blocking=True)
        self.p.resolvent(self.omega, self.n_iter, self.f, self.gains)
        self.gains_host.copy_(self.gains)

    def e2e_bytes(self):
        return self.f_init.numel() * 16, self.P * 8

    def cpu_sample(self, n=64):
        """Oracle: dense R^H G R versus G eigenproblem of the first n pencils (numpy/scipy FP64)."""
        from oracle import couette as oco
        o = oco.Couette(self.Nx, self.Ny, self.Nz, self.Re, pencils=False)
        pairs = [(m, j) for j in range(self.Ny) if j != self.Ny // 2 for m in range(self.Nx // 2)][:n]
        t = time.perf_counter()
        self.oracle_gains = {(m, j): oco.resolvent_gain(o, o.alpha[m], o.beta[j], self.omega) for m, j in pairs}
        el = time.perf_counter() - t
        return n * self.n_iter / el, "%d pencils by the dense generalised eigenproblem, counted as %d iterations " \
            "each" % (n, self.n_iter), el


class KolmogorovMembers(KolmogorovBatch):
    """The batched Kolmogorov workload (same 64 members, observations and horizon) with every
    member as a problem of its own: 64 gradient calls per step, each a persistent launch over one
    member.  Against the batched line this measures what the single mixed-resolution launch gains;
    both compute the same gradient (checked member by member at a 100-step horizon in setup)."""
    name = "kolmogorov2d_members64_mixed128-512_Re100_sbdf2_2000steps_4dvar8"

    def setup(self, device):
        import torch
        from paper_2506_14792_gb300 import spadj
        self.torch, self.sp = torch, spadj
        pack = lambda arrs: np.concatenate([a.ravel() for a in arrs])
        ics = [synthetic.kolmogorov_ic(n, 100 + i) for i, n in enumerate(self.sizes)]
        truths = [synthetic.kolmogorov_ic(n, 5000 + i) for i, n in enumerate(self.sizes)]
        self.x0_host = pack(ics)
        # per-member agreement with the batched launch at a short horizon (same kernels per member)
        self.check = self._compare_with_batch(device, ics, truths, 100)
        self.members, self.x0m, self.gm = [], [], []
        for i, n in enumerate(self.sizes):
            p = spadj.Problem(spadj.SPADJ_KOLMOGOROV2D, spadj.SPADJ_SBDF2, [n], [2 * np.pi], [self.Re, 0.0], self.dt,
                              batch=1)
            p.set_observations(self.obs_steps(), self._obs(p, torch.from_numpy(truths[i].ravel()).to(device),
                                                           self.obs_steps()), 32)
            self.members.append(p)
            self.x0m.append(torch.from_numpy(ics[i].ravel()).to(device))
            self.gm.append(torch.empty_like(self.x0m[-1]))
        self.p = self.members[0]
        self.x0 = torch.from_numpy(self.x0_host).to(device)
        self.x0_pin = torch.from_numpy(self.x0_host).pin_memory()
        self.grad_pin = torch.empty(self.x0.shape, dtype=torch.complex128).pin_memory()
        self.x0_dev2 = torch.empty_like(self.x0)
        self.grad = torch.empty_like(self.x0)

    @staticmethod
    def _obs(p, truth, steps):
        import torch
        out, cur, last = [], truth, 0
        for k in steps:
            nxt = torch.empty_like(cur)
            p.forward(k - last, cur, nxt)
            out.append(nxt)
            cur, last = nxt, k
        return torch.stack(out).contiguous()

    def _compare_with_batch(self, device, ics, truths, nsteps):
        import torch
        sp = self.sp
        k = max(1, nsteps // 8)
        steps = [k * (i + 1) for i in range(8)]
        pack = lambda arrs: torch.from_numpy(np.concatenate([a.ravel() for a in arrs])).to(device)
        pb = sp.Problem(sp.SPADJ_KOLMOGOROV2D, sp.SPADJ_SBDF2, [128], [2 * np.pi], [self.Re, 0.0], self.dt, batch=64,
                        batch_n=self.sizes)
        pb.set_observations(steps, self._obs(pb, pack(truths), steps), 32)
        x0 = pack(ics)
        gb = torch.empty_like(x0)
        pb.gradient(x0, nsteps, gb, objective=sp.SPADJ_OBJ_FOURDVAR)
        worst, off = 0.0, 0
        for i, n in enumerate(self.sizes):
            p = sp.Problem(sp.SPADJ_KOLMOGOROV2D, sp.SPADJ_SBDF2, [n], [2 * np.pi], [self.Re, 0.0], self.dt, batch=1)
            p.set_observations(steps, self._obs(p, torch.from_numpy(truths[i].ravel()).to(device), steps), 32)
            g = torch.empty(ics[i].size, dtype=torch.complex128, device=device)
            p.gradient(torch.from_numpy(ics[i].ravel()).to(device), nsteps, g, objective=sp.SPADJ_OBJ_FOURDVAR)
            ref = gb[off:off + ics[i].size]
            worst = max(worst, float((g - ref).abs().max() / ref.abs().max()))
            off += ics[i].size
            p.close()
        pb.close()
        return {"horizon": nsteps, "max_rel_diff_member_vs_batched": worst}

    def config(self):
        c = KolmogorovBatch.config(self)
        c.update({"workload": self.name, "execution": "64 problems of one member each, gradients called in turn",
                  "vs_batched_launch": self.check})
        return c

    def step(self, ev=None):
        for p, x, g in zip(self.members, self.x0m, self.gm):
            p.gradient(x, self.nsteps, g, objective=self.sp.SPADJ_OBJ_FOURDVAR, want_J=False)

    def forward_step(self):
        for p, x, g in zip(self.members, self.x0m, self.gm):
            p.forward(self.nsteps, x, g)

    def e2e_step(self):
        self.x0_dev2.copy_(self.x0_pin, non_blocking=True)
        off = 0
        for p, x, g in zip(self.members, self.x0m, self.gm):
            n = x.numel()
            p.gradient(self.x0_dev2[off:off + n], self.nsteps, self.grad[off:off + n],
                       objective=self.sp.SPADJ_OBJ_FOURDVAR)
            off += n
        self.grad_pin.copy_(self.grad, non_blocking=True)


class Closure:
    """Learned closure (coarse 64^2 Kolmogorov at Re = 1000 plus the 4-layer 3x3 CNN, 32 channels,
    BF16 operands with FP32 accumulation, FP64 solver) trained through the coarse adjoint on fine
    1024^2 trajectories the solver generates from seeded k^-3 fields (spun up 400 fine steps).
    One bench step = one training iteration: the gradient of the 4D-Var misfit over 128 windows of
    16 coarse steps (dt_c = 4e-3 = 16 fine steps) with respect to the initial states and the CNN
    parameters (spadj_gradient with grad_p), then one Adam step (spadj_adam).  In setup the
    network is trained (150 iterations, model selection on 16 validation windows every 25) and the
    plain coarse, closure and fine solves are timed per window-step and judged on 16 held-out
    windows against the restricted fine solution at T/4, T/2 and T."""
    metric = "closure training window*steps/s through the adjoint (coarse 64^2 + BF16 CNN, FP64 solver)"
    unit = "window*steps/s"
    name = "closure_kolmogorov64_cnn32_Re1000_fine1024_128windows_16steps"
    NF, NC, RE, DTF, RATIO, NCO, SPIN = 1024, 64, 1000.0, 2.5e-4, 16, 16, 400

    def __init__(self, ntrain=128, nval=16, ntest=16, train_iters=150, quick=False):
        self.ntrain, self.nval, self.ntest, self.train_iters = ntrain, nval, ntest, train_iters
        self.quick = quick
        if quick:  # profiling runs: coarse windows of the plain solver, untrained network, no held-out judgement
            self.name = self.name + "_quick"
        self.flush_l2 = False
        self.B = ntrain
        self.dt_c = self.DTF * self.RATIO

    def units_per_step(self):
        return self.ntrain * self.NCO

    def _data(self, seeds):
        import torch
        from paper_2506_14792_gb300 import closure_training as ct
        x0 = torch.from_numpy(np.concatenate([synthetic.kolmogorov_ic(self.NF, s).ravel() for s in seeds])).cuda()
        return ct.make_dataset(x0, len(seeds), self.NF, self.NC, self.RE, self.DTF, self.RATIO, self.NCO,
                               spin=self.SPIN)

    def _per_step_us(self, fn, steps):
        import torch
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return 1e3 * e0.elapsed_time(e1) / steps

    def setup(self, device):
        import torch
        from paper_2506_14792_gb300 import closure_training as ct
        from paper_2506_14792_gb300 import spadj
        self.torch, self.sp, self.ct = torch, spadj, ct
        if self.quick:
            x0 = torch.from_numpy(np.concatenate([synthetic.kolmogorov_ic(self.NC, 1000 + s).ravel()
                                                  for s in range(self.ntrain)])).to(device)
            pp = spadj.Problem(spadj.SPADJ_KOLMOGOROV2D, spadj.SPADJ_SBDF2, [self.NC], [2 * np.pi], [self.RE, 0.0],
                               self.dt_c, batch=self.ntrain)
            self.tr = torch.empty((self.NCO + 1,) + tuple(x0.shape), dtype=x0.dtype, device=device)
            pp.forward(self.NCO, x0, self.tr[-1], self.tr)
            pp.close()
            self.summary = {"setup": "quick: windows of the plain coarse solver as observations, network untrained"}
            self._timed_setup(torch.from_numpy(synthetic.cnn_params(7, scale_out=0.01)).to(device), device)
            return
        t0 = time.perf_counter()
        self.tr = self._data(range(1000, 1000 + self.ntrain))
        va = self._data(range(3000, 3000 + self.nval))
        te = self._data(range(2000, 2000 + self.ntest))
        t_data = time.perf_counter() - t0
        params = torch.from_numpy(synthetic.cnn_params(7, scale_out=0.01)).to(device)
        t0 = time.perf_counter()
        best, hist = ct.train_selected(params, self.tr, self.ntrain, va, self.nval, self.NC, self.RE, self.dt_c,
                                       iters=self.train_iters, every=25, lr=3e-3)
        t_train = time.perf_counter() - t0
        at = [self.NCO // 4, self.NCO // 2, self.NCO]
        zero = torch.zeros_like(best)
        plain = ct.rollout_errors(zero, te, self.ntest, self.NC, self.RE, self.dt_c, at)
        cnn = ct.rollout_errors(best, te, self.ntest, self.NC, self.RE, self.dt_c, at)
        # per window-step costs of the three solvers (forward sweeps over the held-out windows)
        yc = torch.empty_like(te[0])
        pp = spadj.Problem(spadj.SPADJ_KOLMOGOROV2D, spadj.SPADJ_SBDF2, [self.NC], [2 * np.pi], [self.RE, 0.0],
                           self.dt_c, batch=self.ntest)  # the plain coarse solver (no network)
        us_plain = self._per_step_us(lambda: pp.forward(self.NCO, te[0].contiguous(), yc), self.NCO * self.ntest)
        pp.close()
        pc = ct.coarse_problem(self.ntest, self.NC, self.RE, self.dt_c)
        pc.set_params(best)
        us_cnn = self._per_step_us(lambda: pc.forward(self.NCO, te[0].contiguous(), yc), self.NCO * self.ntest)
        pc.close()
        x0f = torch.from_numpy(np.concatenate([synthetic.kolmogorov_ic(self.NF, 2000 + s).ravel()
                                               for s in range(self.ntest)])).to(device)
        pf = spadj.Problem(spadj.SPADJ_KOLMOGOROV2D, spadj.SPADJ_SBDF2, [self.NF], [2 * np.pi], [self.RE, 0.0],
                           self.DTF, batch=self.ntest)
        yf = torch.empty_like(x0f)
        us_fine = self._per_step_us(lambda: pf.forward(self.RATIO * 8, x0f, yf), 8 * self.ntest)
        pf.close()
        mean = lambda d: {("T/4", "T/2", "T")[i]: float(d[k].mean()) for i, k in enumerate(at)}
        self.summary = {
            "held_out_rel_error_vs_fine": {"plain_coarse": mean(plain), "coarse_plus_cnn": mean(cnn)},
            "us_per_window_coarse_step": {"plain_coarse_64": us_plain, "coarse_64_plus_cnn": us_cnn,
                                          "fine_1024_16_fine_steps": us_fine},
            "training": {"iterations": self.train_iters, "validation_history": hist, "train_windows": self.ntrain,
                         "seconds": round(t_train, 1)},
            "data_generation_seconds": round(t_data, 1)}
        self._timed_setup(best, device)

    def _timed_setup(self, params, device):
        """The timed training iteration's problem, optimiser and buffers."""
        torch, ct = self.torch, self.ct
        self.params = params.clone()
        self.p = ct.coarse_problem(self.ntrain, self.NC, self.RE, self.dt_c)
        self.p.set_observations(list(range(1, self.NCO + 1)), self.tr[1:].contiguous(), self.NC // 2 - 1)
        self.opt = ct.Adam(self.p, self.params.numel(), lr=3e-3, device=device)
        self.x0 = self.tr[0].contiguous()
        self.g = torch.empty_like(self.x0)
        self.gp = torch.empty_like(self.params)
        self.x0_pin = self.x0.cpu().pin_memory()
        self.g_pin = torch.empty(self.g.shape, dtype=self.g.dtype).pin_memory()
        self.x0_dev2 = torch.empty_like(self.x0)

    def config(self):
        return {"workload": self.name, "coarse": self.NC, "fine": self.NF, "Re": self.RE, "dt_coarse": self.dt_c,
                "window_steps": self.NCO, "windows": self.ntrain, "cnn": "1-32-32-32-1 3x3 periodic tanh, BF16/FP32",
                "l2": "working set ~%.0f MB (trajectory of the windows), not flushed" % (
                    (self.NCO + 1) * self.ntrain * (self.NC // 2) * self.NC * 16 / 1e6),
                **getattr(self, "summary", {})}

    def step(self, ev=None):
        self.p.set_params(self.params)
        self.p.gradient(self.x0, self.NCO, self.g, objective=self.sp.SPADJ_OBJ_FOURDVAR, grad_p=self.gp, want_J=False)
        self.opt.step(self.params, self.gp)

    def forward_step(self):
        self.p.set_params(self.params)
        self.p.forward(self.NCO, self.x0, self.x0_dev2)

    def e2e_step(self):
        self.x0_dev2.copy_(self.x0_pin, non_blocking=True)
        self.p.set_params(self.params)
        self.p.gradient(self.x0_dev2, self.NCO, self.g, objective=self.sp.SPADJ_OBJ_FOURDVAR, grad_p=self.gp)
        self.opt.step(self.params, self.gp)
        self.g_pin.copy_(self.g, non_blocking=True)

    def e2e_bytes(self):
        n = self.x0.numel() * 16
        return n, n + 8 * self.ntrain

    def cpu_sample(self, n=1, nsteps=16):
        """Oracle: coarse-solver gradient with the FP64 CNN closure (state and parameter gradients)
        of n windows over the full window, numpy FP64."""
        from oracle import cnn as ocnn
        from oracle import imex
        from oracle import kolmogorov as okol
        o = okol.Kolmogorov(self.NC, self.RE, closure=ocnn.CNN(synthetic.cnn_params(7, scale_out=0.01)))
        t = time.perf_counter()
        for s in range(n):
            X0 = o.project(synthetic.kolmogorov_ic(self.NC, 1000 + s))
            target = o.project(synthetic.kolmogorov_ic(self.NC, 3000 + s))
            X = imex.multistep_forward(o, X0, nsteps, self.dt_c)
            imex.multistep_adjoint_params(o, X, lambda k: X[k] - target, self.dt_c)
        el = time.perf_counter() - t
        return n * nsteps / el, "%d windows x %d steps, coarse gradient with the FP64 CNN closure (numpy)" % (
            n, nsteps), el


WORKLOADS = {"burgers": Burgers, "rb": RayleighBenard, "kolmogorov": KolmogorovBatch, "couette": Couette,
             "poiseuille_evp": PoiseuilleEvp, "couette_resolvent": CouetteResolvent,
             "kolmogorov_members": KolmogorovMembers, "closure": Closure}
DEFAULT_WORKLOAD = "rb"


# ---------------------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------------------

def cpu_model():
    """Host CPU model and core count (for the CPU-baseline record)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return model, os.cpu_count()


def _cpu_replica(ctor):
    """One single-threaded oracle sample in a worker process (a fresh workload object)."""
    cls, args, kw = ctor
    wl = cls(*args, **kw)
    v, sample, el = wl.cpu_sample()
    return v, el


def cpu_all_cores(wl):
    """The oracle's throughput on every host core: one independent single-threaded replica of the
    bounded sample per core, run concurrently in spawned processes (the GPU context is never
    forked); value = the replicas' summed units per second."""
    import multiprocessing as mp
    model, n = cpu_model()
    ctor = getattr(wl, "_ctor", (type(wl), (), {}))
    t = time.perf_counter()
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_cpu_replica, [ctor] * n)
    wall = time.perf_counter() - t
    return {"value": float(sum(v for v, _ in res)), "cores": n, "threads_per_replica": 1, "cpu_model": model,
            "replica_seconds": [round(el, 3) for _, el in res], "wall_s": round(wall, 1),
            "note": "%d concurrent single-threaded oracle replicas of the bounded sample" % n}


def reduce_max(x, device=None):
    """Max of a float over all ranks (identity without torch.distributed); gloo or nccl."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank_step, steps, world, ms_max):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank_step * steps * world / (ms_max / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args, wl):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    cores = int(os.environ.get("OPENBLAS_NUM_THREADS", "1"))
    for _ in range(args.warmup):
        wl.cpu_sample()
    vals, secs = [], []
    for _ in range(args.steps):
        v, sample, el = wl.cpu_sample()
        vals.append(v)
        secs.append(el)
    value = float(np.median(vals))
    metric = getattr(wl, "metric", "forward+adjoint gradient dof*steps/s at 1e-10 rel vs FP64 oracle")
    unit = getattr(wl, "unit", "dof*steps/s")
    line = {"impl": "reference", "metric": metric, "value": value,
            "unit": unit, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.median(secs)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": wl.config(),
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gpu(args, wl):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl.setup(dev)
    if args.pdl:
        wl.p.set_option(6, 1)
    if args.no_fuse:
        wl.p.set_option(7, 0)
    if args.x_rows:
        wl.p.set_option(8, args.x_rows)
    if args.host_slots:
        wl.p.set_option(9, args.host_slots)
    for kv in args.set_option:
        k, v = kv.split("=")
        wl.p.set_option(int(k), int(v))
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev) if wl.flush_l2 else None

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()

    for _ in range(args.warmup):
        wl.step()
    barrier()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    for i in range(args.steps):
        if flush is not None:
            flush.fill_(float(i))  # write 256 MB (> L2) between timed iterations, outside the events
        starts[i].record(stream)
        wl.step()
        ends[i].record(stream)
    barrier()
    clocks = clk.stop()
    ms = float(sum(starts[i].elapsed_time(ends[i]) for i in range(args.steps)))
    # adjoint/forward cost ratio: one forward sweep alone (same workload, outside the timed region)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    wl.forward_step()
    barrier()
    f0.record(stream)
    wl.forward_step()
    f1.record(stream)
    barrier()
    fwd_ms = f0.elapsed_time(f1)
    adj_ratio = (ms / args.steps - fwd_ms) / fwd_ms
    # per-kernel breakdown: one more step of the same workload with the library bracketing each
    # of its launches by CUDA events on this stream (kept out of the timed region: the events
    # add host work between launches)
    wl.p.timing(True)
    if flush is not None:
        flush.fill_(-1.0)
    wl.step()
    barrier()
    rep = wl.p.timing_report()
    wl.p.timing(False)
    ms = reduce_max(ms, dev)
    units = wl.units_per_step() * args.steps * ws
    value = job_value(wl.units_per_step(), args.steps, ws, ms)

    # end to end through the public API with host buffers
    for _ in range(max(1, args.warmup // 2)):
        wl.e2e_step()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        wl.e2e_step()
    e1.record(stream)
    barrier()
    e2e_ms = reduce_max(e0.elapsed_time(e1), dev)
    bi, bo = wl.e2e_bytes()

    # roofline of the dominant kernel class (FP64 ALU bound on GB300) against the measured FP64 peak
    fp64 = measure_fp64_peak(local)
    peak = fp64["gflops"]
    dom = max(rep, key=lambda k: rep[k][0])
    dms, dfl, dn = rep[dom]
    achieved = dfl / (dms / 1e3) / 1e9
    per_kernel = {k: {"ms_total": v[0], "launches": v[2], "share": v[0] / sum(x[0] for x in rep.values()),
                      "gflops": v[1] / (v[0] / 1e3) / 1e9 if v[0] > 0 else None} for k, v in rep.items()}
    # the FP64 classes only: a class on the BF16 tensor cores (the closure network) has its own roof
    total_flops = sum(v[1] for k, v in rep.items() if k != "cnn")
    bound, dpeak, psrc = "alu", peak, "measured"
    if dom == "cnn":  # BF16 operands on the tensor cores: the measured dense BF16 rate
        bound = "tensor"
        dpeak, psrc = bf16_peak_gflops()
    roof = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": dpeak, "unit": "GFLOP/s",
            "frac": achieved / dpeak, "traffic": traffic_for(wl, dom),
            "hbm": hbm_fraction(traffic_for(wl, dom), dms / dn / 1e3),
            "avg_launch_us": 1e3 * dms / dn, "flops_per_launch": dfl / dn, "per_kernel": per_kernel,
            "whole_step": {"algorithmic_gflop": total_flops / 1e9,
                           "achieved": total_flops / (ms / args.steps / 1e3) / 1e9,
                           "frac": total_flops / (ms / args.steps / 1e3) / 1e9 / peak,
                           "note": "all FP64 kernel classes' algorithmic flops of one step over the timed step"
                                   + (" (the closure network's BF16 tensor-core class excluded)" if "cnn" in rep else "")},
            "peak_source": psrc, "peak_measurement": fp64 if bound == "alu" else "MEASURED_PEAKS.json bf16_tflops",
            "peak_note": "FP64 peak measured by the library's FMA-chain probe on this GPU (nominal %.0f GFLOP/s = "
                         "152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz); no tensor-core FP64 path (GB300's FP64 "
                         "tensor rate is the same). Per-class times come from one instrumented step in which "
                         "the reverse sweep's lanes overlap, so each class's GFLOP/s is a lower bound"
                         % FP64_NOMINAL_GFLOPS}
    launches = int(sum(v[2] for v in rep.values())) * args.steps
    if rank != 0:
        return 0
    cpu = None
    if ws == 1 and not args.no_cpu:
        v, sample, el = wl.cpu_sample()
        model, _ = cpu_model()
        cpu = {"value": v, "unit": getattr(wl, "unit", "dof*steps/s"), "cores": int(os.environ.get("OPENBLAS_NUM_THREADS", "1")),
               "kind": "oracle", "sample": sample, "cpu_model": model}
        if not args.no_cpu_all:
            cpu["all_cores"] = cpu_all_cores(wl)
    line = {"metric": getattr(wl, "metric", "forward+adjoint gradient dof*steps/s at 1e-10 rel vs FP64 oracle"),
            "value": value,
            "unit": getattr(wl, "unit", "dof*steps/s"), "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": dict(wl.config(), parallelism="replicas%d" % ws,
                           **({"host_checkpoint_slots": args.host_slots} if args.host_slots else {}),
                           **({"options": args.set_option} if args.set_option else {})),
            "gpu_launches": launches,
            "e2e": {"value": units / (e2e_ms / 1e3), "unit": getattr(wl, "unit", "dof*steps/s"),
                    "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo},
            "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
            "adjoint_forward_ratio": {"value": adj_ratio, "forward_ms": fwd_ms,
                                      "definition": "(gradient - forward sweep) / forward sweep, same workload"}}
    print(json.dumps(line))
    return 0


def run_gpu_evp(args, wl):
    """Bench line of the eigenvalue workload: value from the library's CUDA events around its
    kernels (operators resident on the device), e2e from the whole spadj_eigen call (host
    factorisation, operator upload, iterations, result read-back)."""
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl.setup(dev)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()

    for _ in range(args.warmup):
        wl.step()
    barrier()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    wl.p.timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        wl.step()
    e1.record(stream)
    barrier()
    clocks = clk.stop()
    rep = wl.p.timing_report()
    wl.p.timing(False)
    dev_ms = reduce_max(float(sum(v[0] for v in rep.values())), dev)
    e2e_ms = reduce_max(e0.elapsed_time(e1), dev)
    units = wl.units_per_step() * args.steps * ws
    value = job_value(wl.units_per_step(), args.steps, ws, dev_ms)
    evp = isinstance(wl, PoiseuilleEvp)
    extra = {}
    if evp:
        o = wl.out.cpu().numpy()
        extra["converged_fraction"] = float(np.mean(np.max(o[:, 8:10], axis=1) <= 1e-11))
        dom = "pencil_solve"
    else:
        g = wl.gains_host.numpy()
        extra["gain_range"] = [float(g[g > 0].min()), float(g.max())]
        dom = max(rep, key=lambda k: rep[k][0])
        # the GPU gains of the pencils the CPU oracle solves (dense generalised eigenproblem)
        if rank == 0:
            if ws == 1 and not args.no_cpu:
                wl.cpu_result = wl.cpu_sample()  # the CPU baseline leg (reported below)
            else:
                wl.cpu_sample(n=16)
            err = np.array([abs(g[j, m] - v) / v for (m, j), v in wl.oracle_gains.items()])
            extra["vs_oracle"] = {"pencils": int(err.size), "max_rel_err": float(err.max()),
                                  "within_1e-10": float(np.mean(err <= 1e-10)),
                                  "within_1e-6": float(np.mean(err <= 1e-6)),
                                  "note": "%d power iterations from a random forcing; the oracle is the converged "
                                          "leading gain" % wl.n_iter}
    dms, dfl, dn = rep[dom]
    achieved = dfl / (dms / 1e3) / 1e9
    fp64 = measure_fp64_peak(local)
    peak = fp64["gflops"]
    per_kernel = {k: {"ms_total": v[0], "launches": v[2], "share": v[0] / sum(x[0] for x in rep.values()),
                      "gflops": v[1] / (v[0] / 1e3) / 1e9 if v[0] > 0 else None} for k, v in rep.items()}
    roof = {"kernel": "evp_iter_kernel (pencil_solve)" if evp else dom, "bound": "alu", "achieved": achieved,
            "peak": peak, "unit": "GFLOP/s", "frac": achieved / peak, "peak_source": "measured",
            "peak_measurement": fp64,
            "traffic": traffic_for(wl, dom), "hbm": hbm_fraction(traffic_for(wl, dom), dms / dn / 1e3),
            "avg_launch_us": 1e3 * dms / dn, "flops_per_launch": dfl / dn,
            "per_kernel": per_kernel,
            "peak_note": "FP64 peak measured by the library's FMA-chain probe on this GPU; "
                         + ("16 flops per operator entry and iteration (forward and adjoint complex matvecs)" if evp
                            else "8 flops per operator entry and pencil solve (complex matvec), 4 per entry of "
                                 "the real Gram products")}
    launches = int(sum(v[2] for v in rep.values()))
    if rank != 0:
        return 0
    cpu = None
    if ws == 1 and not args.no_cpu:
        v, sample, el = getattr(wl, "cpu_result", None) or wl.cpu_sample()
        model, _ = cpu_model()
        cpu = {"value": v, "unit": wl.unit, "cores": int(os.environ.get("OPENBLAS_NUM_THREADS", "1")),
               "kind": "oracle", "sample": sample, "cpu_model": model}
        if not args.no_cpu_all:
            cpu["all_cores"] = cpu_all_cores(wl)
    bi, bo = wl.e2e_bytes()
    line = {"metric": wl.metric, "value": value, "unit": wl.unit, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(wl.config(), parallelism="replicas%d" % ws, **extra),
            "gpu_launches": launches,
            "e2e": {"value": units / (e2e_ms / 1e3), "unit": wl.unit, "h2d_bytes_per_step": bi,
                    "d2h_bytes_per_step": bo,
                    "note": "includes the host LU of every shifted pencil" if evp else
                            "the frequency's pencil factorisations are built at the first call and kept"},
            "roofline": roof, "cpu_baseline": cpu, "clocks": clocks}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--no-cpu-all", action="store_true", help="skip the all-cores CPU-oracle replicas")
    ap.add_argument("--pdl", action="store_true", help="programmatic dependent launch of consecutive kernels")
    ap.add_argument("--no-fuse", action="store_true", help="RB: separate fold / solve / expand kernels")
    ap.add_argument("--x-rows", type=int, default=0, help="x-FFT rows per CTA (1, 2, 4; 0 = tuned)")
    ap.add_argument("--host-slots", type=int, default=0,
                    help="rb/couette: host checkpoint slots (two-level schedule; device slots then from --hbm-gb)")
    ap.add_argument("--hbm-gb", type=float, default=None, help="couette: device checkpoint budget in GB")
    ap.add_argument("--set-option", action="append", default=[], metavar="K=V",
                    help="spadj_set_option(K, V) on the workload's problem before the run (repeatable)")
    ap.add_argument("--nsteps", type=int, default=None,
                    help="override the workload's time steps, or the iterations of poiseuille_evp (profiling runs)")
    ap.add_argument("--size", default=None,
                    help="override the grid of the rb (Nx,Nz) or couette (Nx,Ny,Nz) workload, or the pencil "
                         "grid (n_alpha,n_beta) of poiseuille_evp (profiling runs)")
    ap.add_argument("--scheme", default=None,
                    help="rb: rk222 (default) or rk443; burgers: sbdf1..sbdf4 (default sbdf2)")
    ap.add_argument("--op", default=None, choices=["gain", "integral", "hvp"],
                    help="couette: gain gradient (default), time-integrated energy gradient, or Hessian-vector product")
    ap.add_argument("--omega", type=float, default=None, help="couette_resolvent: forcing frequency (default 0)")
    ap.add_argument("--batch", type=int, default=None,
                    help="burgers: members per gradient (default 16384; 1 gives the single-member latency line)")
    ap.add_argument("--quick", action="store_true",
                    help="closure: skip the fine data and the training (profiling runs; same timed iteration)")
    ap.add_argument("--slots", type=int, default=0,
                    help="burgers: binomial checkpointing with this many restart-state slots; kolmogorov: this many "
                         "checkpointed segments (0: store-all)")
    ap.add_argument("--dt-blocks", type=int, default=0,
                    help="rb: step-size schedule alternating dt and dt/2 every this many steps (0: constant dt)")
    args = ap.parse_args()
    kw = {}
    if args.scheme is not None:
        ok = {"rb": ("rk222", "rk443"), "burgers": tuple(Burgers.ORDERS)}.get(args.workload, ())
        if args.scheme not in ok:
            ap.error("--scheme %s does not apply to the %s workload" % (args.scheme, args.workload))
        kw["scheme"] = args.scheme
    if args.op is not None:
        if args.workload != "couette":
            ap.error("--op applies to the couette workload")
        kw["op"] = args.op
    if args.nsteps is not None:
        if args.workload == "couette_resolvent":
            kw["n_iter"] = args.nsteps
        elif args.workload != "poiseuille_evp":
            kw["nsteps"] = args.nsteps
    if args.dt_blocks:
        if args.workload != "rb":
            ap.error("--dt-blocks applies to the rb workload")
        kw["dt_blocks"] = args.dt_blocks
    if args.batch is not None:
        if args.workload != "burgers" or args.batch < 1:
            ap.error("--batch (>= 1) applies to the burgers workload")
        kw["batch"] = args.batch
    if args.quick:
        if args.workload != "closure":
            ap.error("--quick applies to the closure workload")
        kw["quick"] = True
    if args.slots:
        if args.workload not in ("burgers", "kolmogorov") or args.slots < 1:
            ap.error("--slots (>= 1) applies to the burgers and kolmogorov workloads")
        kw["slots"] = args.slots
    if args.omega is not None:
        if args.workload != "couette_resolvent":
            ap.error("--omega applies to the couette_resolvent workload")
        kw["omega"] = args.omega
    wl = WORKLOADS[args.workload](**kw)
    wl._ctor = (type(wl), (), dict(kw))
    if args.nsteps is not None:
        wl.nsteps = args.nsteps
    if args.workload == "poiseuille_evp" and (args.nsteps is not None or args.size):
        dims = [int(v) for v in args.size.split(",")] if args.size else [38, 16]
        if len(dims) != 2:
            ap.error("--size takes n_alpha,n_beta for poiseuille_evp")
        it = args.nsteps if args.nsteps is not None else wl.n_iter
        wl = PoiseuilleEvp(n_alpha=dims[0], n_beta=dims[1], n_iter=it)
        wl.name = "poiseuille_evp_N64_%dpencils_Re8000_%diter" % (wl.P, it)
        wl._ctor = (PoiseuilleEvp, (), {"n_alpha": dims[0], "n_beta": dims[1], "n_iter": it})
    elif args.size:
        dims = [int(v) for v in args.size.split(",")]
        if args.workload == "couette" and len(dims) == 3:
            wl = Couette(*dims, **kw)
            wl._ctor = (Couette, tuple(dims), dict(kw))
            wl.name = "couette3d_%dx%dx%d_Re1000_sbdf2_%dsteps_%s" % (dims[0], dims[1], dims[2], wl.nsteps, wl.op)
        elif args.workload == "couette_resolvent" and len(dims) == 3:
            wl = CouetteResolvent(*dims, **kw)
            wl._ctor = (CouetteResolvent, tuple(dims), dict(kw))
        elif args.workload == "rb" and len(dims) == 2:
            wl = RayleighBenard(*dims, **kw)
            wl._ctor = (RayleighBenard, tuple(dims), dict(kw))
        else:
            ap.error("--size takes Nx,Nz for rb and Nx,Ny,Nz for couette and couette_resolvent")
    if args.hbm_gb is not None:
        if not isinstance(wl, Couette):
            ap.error("--hbm-gb applies to the couette workload")
        wl.budget = args.hbm_gb * 1e9
    if args.impl == "reference":
        return run_reference(args, wl)
    if isinstance(wl, (PoiseuilleEvp, CouetteResolvent)):
        return run_gpu_evp(args, wl)
    return run_gpu(args, wl)


if __name__ == "__main__":
    sys.exit(main())
