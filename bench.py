"""Benchmark: forward+adjoint gradient evaluations in dof*steps/s.

One bench "step" is one whole gradient evaluation of the workload (forward sweep with
checkpoint/trajectory writes, objective, adjoint sweep) over one batch of synthetic
input resident in HBM.  The GPU arm runs the CUDA library through its C-ABI; the
reference arm (``--impl reference``) times the FP64 CPU oracle on a bounded sample of
the same workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                       [--workload rb|burgers]
Under torchrun (N > 1) each rank runs an independent replica / shard; the time is the
max over ranks and the value counts the units of all ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 peak: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz (nominal GB300 FP64 1.25 TFLOP/s).
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07


def fp64_flops_real_fft(M):
    """Conventional flop count of one real FFT of length M (half of 5 M log2 M)."""
    return 2.5 * M * np.log2(M)


# ---------------------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------------------

class Burgers:
    """1D viscous Burgers, N=256, nu=0.01, SBDF2 dt=1e-3, 1000 steps, 16384 members."""
    name = "burgers1d_N256_sbdf2_1000steps"

    def __init__(self, batch=16384, N=256, nsteps=1000, dt=1e-3, nu=0.01, seed=1):
        self.B, self.N, self.nsteps, self.dt, self.nu, self.seed = batch, N, nsteps, dt, nu, seed
        self.dof = N
        self.K, self.M = N // 2, 3 * N // 2

    def config(self):
        return {"workload": self.name, "N": self.N, "nu": self.nu, "dt": self.dt, "steps": self.nsteps,
                "batch": self.B, "scheme": "SBDF2", "objective": "0.5||u(T)||^2",
                "l2": "working set > L2 (stored trajectory %.1f GB)" % (self.traj_bytes() / 1e9)}

    def traj_bytes(self):
        return (self.nsteps + 1) * self.B * self.K * 16

    def units_per_step(self):
        return self.B * self.dof * self.nsteps

    # algorithmic FP64 flops per member per step: 2 real FFTs forward, 3 adjoint (+ pointwise)
    def kernel_flops(self):
        f = fp64_flops_real_fft(self.M)
        fwd = self.B * self.nsteps * (2 * f + self.M + 10 * self.K)
        adj = self.B * self.nsteps * (3 * f + 2 * self.M + 12 * self.K)
        return {"forward": fwd, "adjoint": adj}

    def setup(self, device):
        import torch
        from paper_2506_14792_gb300 import spadj
        self.torch = torch
        self.sp = spadj
        self.p = spadj.Problem(spadj.SPADJ_BURGERS1D, spadj.SPADJ_SBDF2, [self.N], [2 * np.pi], [self.nu], self.dt,
                               batch=self.B)
        self.X0_host = synthetic.burgers_ic(self.N, batch=self.B, seed=self.seed)
        self.x0 = torch.from_numpy(self.X0_host).to(device)
        self.traj = torch.empty((self.nsteps + 1, self.B, self.K), dtype=torch.complex128, device=device)
        self.xN = self.traj[-1]
        self.J = torch.empty(self.B, dtype=torch.float64, device=device)
        self.seedv = torch.empty((self.B, self.K), dtype=torch.complex128, device=device)
        self.grad = torch.empty((self.B, self.K), dtype=torch.complex128, device=device)
        self.x0_pin = torch.from_numpy(self.X0_host).pin_memory()
        self.grad_pin = torch.empty((self.B, self.K), dtype=torch.complex128).pin_memory()
        self.x0_dev2 = torch.empty_like(self.x0)

    def launches_per_step(self):
        return 3

    def step(self, ev):
        """Device-resident step; ev = list of 4 events recorded between the kernels."""
        ev[0].record()
        self.p.forward(self.nsteps, self.x0, self.xN, self.traj)
        ev[1].record()
        self.p.objective(self.xN, self.J, self.seedv)
        ev[2].record()
        self.p.adjoint(self.nsteps, self.traj, self.seedv, self.grad)
        ev[3].record()

    def kernel_names(self):
        return ["forward", "objective", "adjoint"]

    def e2e_step(self):
        """Public API call with host buffers: pinned H2D of x0, spadj_gradient (J to host), D2H of grad."""
        self.x0_dev2.copy_(self.x0_pin, non_blocking=True)
        J = self.p.gradient(self.x0_dev2, self.nsteps, self.grad)
        self.grad_pin.copy_(self.grad, non_blocking=True)
        return J

    def e2e_bytes(self):
        return self.B * self.K * 16, self.B * self.K * 16 + self.B * 8

    # CPU oracle on a bounded sample
    def cpu_sample(self):
        from oracle import burgers as ob
        o = ob.Burgers(self.N, self.nu)
        Bs = 256
        X0 = self.X0_host[:Bs] if hasattr(self, "X0_host") else synthetic.burgers_ic(self.N, batch=Bs, seed=self.seed)
        t = time.perf_counter()
        ob.gradient(o, X0, self.nsteps, self.dt)
        el = time.perf_counter() - t
        return Bs * self.dof * self.nsteps / el, "%d members x %d steps (gradient, numpy FP64)" % (Bs, self.nsteps), el


WORKLOADS = {"burgers": Burgers}
DEFAULT_WORKLOAD = "burgers"


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

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args, wl):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    cores = int(os.environ.get("OMP_NUM_THREADS", "1"))
    for _ in range(args.warmup):
        wl.cpu_sample()
    vals, secs = [], []
    for _ in range(args.steps):
        v, sample, el = wl.cpu_sample()
        vals.append(v)
        secs.append(el)
    value = float(np.median(vals))
    line = {"impl": "reference", "metric": "forward+adjoint gradient dof*steps/s (FP64 oracle, CPU)", "value": value,
            "unit": "dof*steps/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.median(secs)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": wl.config(),
            "cpu_baseline": {"value": value, "unit": "dof*steps/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "dof*steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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
    stream = torch.cuda.current_stream()
    names = wl.kernel_names()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)] for _ in range(args.steps)]
    warm = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
    for _ in range(args.warmup):
        wl.step(warm)
    barrier()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        wl.step(evs[i])
    t1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = t0.elapsed_time(t1)
    per_kernel = {nm: float(np.mean([evs[i][j].elapsed_time(evs[i][j + 1]) for i in range(args.steps)]))
                  for j, nm in enumerate(names)}
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    units = wl.units_per_step() * args.steps * ws
    value = units / (ms / 1e3)

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
    e2e_ms = e0.elapsed_time(e1)
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    bi, bo = wl.e2e_bytes()

    # roofline of the dominant kernel (FP64 ALU bound)
    flops = wl.kernel_flops()
    dom = max(flops, key=lambda k: per_kernel.get(k, 0.0))
    achieved = flops[dom] / (per_kernel[dom] / 1e3) / 1e9
    roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
            "frac": achieved / FP64_PEAK_GFLOPS, "traffic": wl.traffic(dom) if hasattr(wl, "traffic") else None,
            "per_kernel_ms": per_kernel,
            "peak_note": "FP64 FMA peak 152 SM x 2 DFMA/clk x 2.07 GHz (nominal 1.25 TFLOP/s)"}
    if rank != 0:
        return 0
    cpu = None
    if ws == 1 and not args.no_cpu:
        v, sample, el = wl.cpu_sample()
        cpu = {"value": v, "unit": "dof*steps/s", "cores": 1, "kind": "oracle", "sample": sample}
    line = {"metric": "forward+adjoint gradient dof*steps/s at 1e-10 rel vs FP64 oracle", "value": value,
            "unit": "dof*steps/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": dict(wl.config(), parallelism="dp%d" % ws),
            "gpu_launches": wl.launches_per_step() * args.steps,
            "e2e": {"value": units / (e2e_ms / 1e3), "unit": "dof*steps/s", "h2d_bytes_per_step": bi,
                    "d2h_bytes_per_step": bo},
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
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]()
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_gpu(args, wl)


if __name__ == "__main__":
    sys.exit(main())
