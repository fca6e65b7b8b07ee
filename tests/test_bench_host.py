"""Host logic of bench.py's roofline fields (no GPU): the DRAM traffic reported for a kernel
whose traffic is its stored trajectory scales with the run's horizon, horizon-independent
entries do not, uncaptured workloads report None, and the HBM fraction divides the traffic by
the launch time and the measured copy bandwidth."""
import sys

import pytest


@pytest.fixture(scope="module")
def bench():
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        import bench as b
    finally:
        sys.argv = argv
    return b


def test_trajectory_traffic_scales_with_stored_steps(bench):
    w = bench.Burgers()
    full = bench.traffic_for(w, "fused_trajectory")
    assert full == bench.TRAFFIC[(w.name, "fused_trajectory")]
    w.nsteps = 50
    assert bench.traffic_for(w, "fused_trajectory") == pytest.approx(full * 51 / 1001, rel=1e-15)


def test_per_launch_traffic_is_horizon_independent(bench):
    r = bench.RayleighBenard()
    t = bench.traffic_for(r, "x_fft")
    r.nsteps = 4
    assert bench.traffic_for(r, "x_fft") == t == bench.TRAFFIC[(r.name, "x_fft")]
    assert bench.traffic_for(r, "no_such_kernel") is None
    k = bench.KolmogorovBatch()  # not captured on the gradient's sweeps: reported as null
    assert bench.traffic_for(k, "fused_trajectory") is None


def test_hbm_fraction(bench):
    h = bench.hbm_fraction(6.0e9, 2.0e-3)  # 6 GB in 2 ms
    assert h["achieved_gbs"] == pytest.approx(3000.0)
    assert h["frac"] == pytest.approx(3000.0 / h["peak_gbs"])
    assert bench.hbm_fraction(None, 2.0e-3) is None


@pytest.mark.parametrize("argv,name,check", [
    (["--workload", "rb", "--scheme", "rk443", "--nsteps", "200"], "rayleigh_benard2d_256x64_Ra1e6_rk443_200steps",
     lambda w: w.scheme == "rk443" and w.nsteps == 200),
    (["--workload", "rb", "--dt-blocks", "50", "--nsteps", "200"],
     "rayleigh_benard2d_256x64_Ra1e6_rk222_200steps_dtblocks50",
     lambda w: w.schedule()[49] == w.dt and w.schedule()[50] == 0.5 * w.dt and len(w.schedule()) == 200),
    (["--workload", "rb", "--size", "128,32", "--dt-blocks", "50", "--nsteps", "200"],
     "rayleigh_benard2d_128x32_Ra1e6_rk222_200steps_dtblocks50",
     lambda w: w.Nx == 128 and w.Nz == 32 and w.dt_blocks == 50 and len(w.schedule()) == 200),
    (["--workload", "burgers", "--batch", "1"], "burgers1d_N256_sbdf2_1000steps_b1",
     lambda w: w.B == 1 and w.units_per_step() == 256 * 1000),
    (["--workload", "burgers", "--scheme", "sbdf4"], "burgers1d_N256_sbdf4_1000steps",
     lambda w: w.ORDERS[w.scheme] == 4),
    (["--workload", "couette", "--op", "hvp", "--size", "64,32,32", "--nsteps", "100"],
     "couette3d_64x32x32_Re1000_sbdf2_100steps_hvp", lambda w: w.op == "hvp" and "Hessian" in w.metric),
    (["--workload", "couette_resolvent", "--nsteps", "20", "--omega", "0.3"],
     "couette3d_64x32x32_Re1000_resolvent_omega0.3_20iter", lambda w: w.units_per_step() == 1024 * 20),
    ([], "rayleigh_benard2d_256x64_Ra1e6_rk222_2000steps", lambda w: w.scheme == "rk222" and not w.dt_blocks),
    (["--workload", "burgers", "--slots", "32"], "burgers1d_N256_sbdf2_1000steps_ckpt32",
     lambda w: w.slots == 32 and "binomial" in w.config()["checkpointing"]),
    (["--workload", "kolmogorov", "--slots", "40"], "kolmogorov2d_batch64_mixed128-512_Re100_sbdf2_2000steps_4dvar8_seg40",
     lambda w: w.slots == 40 and "segments" in w.config()["checkpointing"]),
    (["--workload", "closure", "--quick"], "closure_kolmogorov64_cnn32_Re1000_fine1024_128windows_16steps_quick",
     lambda w: w.quick and w.units_per_step() == 128 * 16),
])
def test_workload_variants_from_the_command_line(bench, argv, name, check):
    """The variant flags build the workload they name (the run itself is replaced by a probe)."""
    got = []
    run_gpu, run_gpu_evp, saved = bench.run_gpu, bench.run_gpu_evp, sys.argv
    bench.run_gpu = bench.run_gpu_evp = lambda args, wl: got.append(wl) or 0
    sys.argv = ["bench.py"] + argv
    try:
        assert bench.main() == 0
    finally:
        bench.run_gpu, bench.run_gpu_evp, sys.argv = run_gpu, run_gpu_evp, saved
    assert got[0].name == name and check(got[0])


@pytest.mark.parametrize("argv", [["--workload", "burgers", "--dt-blocks", "5"],
                                  ["--workload", "rb", "--batch", "4"],
                                  ["--workload", "rb", "--scheme", "sbdf2"],
                                  ["--workload", "rb", "--op", "hvp"],
                                  ["--workload", "couette", "--omega", "1.0"],
                                  ["--workload", "rb", "--slots", "8"],
                                  ["--workload", "burgers", "--quick"]])
def test_variant_flags_refused_where_they_do_not_apply(bench, argv):
    saved = sys.argv
    sys.argv = ["bench.py"] + argv
    try:
        with pytest.raises(SystemExit):
            bench.main()
    finally:
        sys.argv = saved
