"""Writes rb_256x64_ra1e6_rk222_2000steps.npz: the oracle's kinetic energy at T and its
gradient with respect to the initial state for the full Rayleigh-Benard configuration
(Fourier 256 x Chebyshev 64, Ra = 1e6, Pr = 1, RK222 (ARS(2,2,2)), dt = 1e-3, 2000 steps,
initial state synthetic.rb_ic(256, 64, seed=2, amp=1e-3)), computed by the discrete RK
adjoint of Supplementary A.4 over the stored trajectory ("Efficiently calculating gradients",
eqs. 1-6).

The oracle is run twice: once with numpy's FFT for the x transforms and once with direct
sums over explicit exponentials (the same maps summed in another order).  The difference of
the two runs is the oracle's own rounding-order spread at this horizon; a parity test of
another implementation against the stored values cannot be tighter than that.  Stored:

  J, grad            -- FFT run (the reference values; grad in the state layout (3, 128, 64))
  J_direct, grad_direct -- direct-sum run
  spread_steps, spread_state -- max-norm relative difference of the two forward states at
                        every 100th step
  spread_J, spread_grad -- relative differences of J and (max-norm) of the gradients

Only oracle/ and the seeded input generator are used.  Run from the repository root:
    python tests/golden/make_rb_256x64_2000steps.py      (about 30 min on 2 x 3 cores)
"""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rb_256x64_ra1e6_rk222_2000steps.npz")
NX, NZ, RA, DT, NSTEPS = 256, 64, 1e6, 1e-3, 2000


def _run(x_sums):
    sys.path.insert(0, ROOT)
    import synthetic
    from oracle import rayleigh_benard as orb
    o = orb.RayleighBenard(NX, NZ, RA, x_sums=x_sums)
    s0 = synthetic.rb_ic(NX, NZ, seed=2, amp=1e-3)
    J, g, X, _ = orb.gradient(o, o.pencils(s0), NSTEPS, DT)
    states = np.stack([o.state(X[n]) for n in range(0, NSTEPS + 1, 100)])
    return float(J), o.state(g), states


def main():
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "3")
    ctx = mp.get_context("spawn")
    with ctx.Pool(2) as pool:
        (J, g, st), (Jd, gd, std) = pool.map(_run, ["fft", "direct"])
    rel = lambda a, b: float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    steps = np.arange(0, NSTEPS + 1, 100)
    spread_state = np.array([rel(std[i], st[i]) if np.max(np.abs(st[i])) > 0 else 0.0 for i in range(len(steps))])
    np.savez(OUT, J=J, grad=g, J_direct=Jd, grad_direct=gd, spread_steps=steps, spread_state=spread_state,
             spread_J=abs(Jd - J) / abs(J), spread_grad=rel(gd, g))
    print("J", J, "spread_J", abs(Jd - J) / abs(J), "spread_grad", rel(gd, g))
    print("state spread by step:", dict(zip(steps.tolist(), spread_state.tolist())))


if __name__ == "__main__":
    main()
