"""Host-side pieces of bench.py that need no GPU: the algorithmic counts and the roofline objects it
assembles from kernel timings (so that a missing capture or an odd timing dict cannot break the JSON
line)."""
import bench


def test_scaled_traffic_handles_missing_captures():
    assert bench.scaled_traffic(None, 100) is None
    assert bench.scaled_traffic(10.0, 100) == 1000.0
    assert bench.scaled_traffic(10.0, 100, applies=False) is None


def test_fp32_step_roofline_from_kernel_timings():
    kt = {"face": (1.5, 10), "lift": (3.9, 10), "volume": (10.3, 10), "other": (0.3, 1), "indicator": (0.0, 0)}
    r = bench.fp32_step_roofline(7, 32768, kt, region_ms=16.0)
    assert r["bound"] == "hbm" and 0.0 < r["frac"] < 2.0
    assert set(r["kernels"]) == {"face", "lift", "volume", "other"}
    per = bench.fp32_kernel_bytes_per_launch(7, 32768)
    total = sum(per[k] * kt[k][1] for k in per)
    assert abs(r["achieved"] - total / 16e-3 / 1e9) < 1e-6 * r["achieved"]
    assert r["bytes_per_step"] == total / 2  # 10 volume launches = 2 steps of 5 stages


def test_algorithmic_counts_are_positive_and_grow_with_degree():
    for f in (lambda N: bench.volume_kernel_flops_per_element(N, True), bench.lift_kernel_flops_per_element,
              bench.adjoint_visc_flops_per_element, lambda N: bench.fv_subcell_flops_per_element(N, bench.LLF_FLOPS),
              lambda N: bench.adjoint_volume_flops_per_element(N, True)):
        vals = [f(N) for N in range(1, 8)]
        assert all(v > 0 for v in vals) and vals == sorted(vals)
    assert bench.volume_kernel_bytes_per_element(7, True, 4) < bench.volume_kernel_bytes_per_element(7, True, 8)
