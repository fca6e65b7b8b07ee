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
