"""Host logic of bench.py's JSON line that needs no GPU: the dominant-kernel
roofline built from per-launch unit timings."""
import pytest

import bench


def test_kernel_roofline_picks_the_dominant_unit_and_counts_algorithmic_bytes():
    N, M, B, steps = 256, 64, 64, 10
    L = N * N * M
    # 32 launches of 2 problems per unit per step
    stats = [(0.030 * 320, 320), (0.032 * 320, 320), (0.027 * 320, 320)]
    r = bench.kernel_roofline(stats, N, M, B, steps, 6780.7, "measured", 2100.0, B * 12 * L, "f32")
    assert r["kernel"] == "kf_lines"
    assert r["alg_bytes_per_launch"] == 2 * 8 * M * N * (N // 2 + 1)
    assert r["avg_launch_ms"] == pytest.approx(0.032)
    assert r["achieved"] == pytest.approx(r["alg_bytes_per_launch"] / 0.032e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6780.7)
    assert r["traffic"] == pytest.approx((71.606432 + 0.042944) * 1e6)
    assert r["traffic_warm_cache"] == pytest.approx((36.260768 + 6.264480) * 1e6)
    # warm-cache traffic of the whole step: 1.33x the algorithmic 12 bytes per point
    assert r["step"]["traffic_warm_cache"] / (12 * L) == pytest.approx(1.33, abs=0.01)
    assert [k["kernel"] for k in r["kernels"]] == ["kf_fwd_xt", "kf_lines", "kf_inv_tx"]
    assert r["kernels"][0]["alg_bytes_per_launch"] == 2 * 4 * L
    assert r["step"]["achieved"] == 2100.0


def test_kernel_roofline_half_rows_and_other_group_sizes_drop_the_ncu_traffic():
    N, M, B, steps = 256, 64, 48, 1
    stats = [(1.0, 16), (2.0, 16), (1.0, 16)]          # 3 problems per launch
    r = bench.kernel_roofline(stats, N, M, B, steps, 6780.7, "measured", 1.0, 1.0, "f32")
    assert r["traffic"] is None
    stats = [(1.0, 24), (2.0, 24), (1.0, 24)]          # 2 problems per launch, half the C rows
    r = bench.kernel_roofline(stats, N, M, B, steps, 6780.7, "measured", 1.0, 1.0, "f32", c_rows=N // 2 + 1)
    assert r["traffic"] is None and r["traffic_warm_cache"] is None
    assert r["alg_bytes_per_launch"] == 2 * 8 * M * (N // 2 + 1) * (N // 2 + 1)


def test_kernel_roofline_without_unit_timings_reports_the_step():
    r = bench.kernel_roofline([(0.0, 0)] * 3, 512, 128, 8, 5, 6780.7, "measured", 1234.0, 8 * 12.0, "split_bf16")
    assert r["achieved"] == 1234.0 and r["scope"].startswith("whole")


def test_grid_flops_counts_the_six_passes():
    # one real x-forward line costs 4 Lx (Kx + 1) flops, and so on; at L = N = (3, 3, 3), Kx = 1
    assert bench.grid_flops((3, 3, 3), (3, 3, 3), k=0) == (4 * 3 * 3 * 2 * 3 + 8 * 3 * 2 * 3 * 3 + 8 * 3 * 2 * 3 * 3
                                                          + 8 * 3 * 2 * 3 * 3 + 8 * 3 * 2 * 3 * 3 + 4 * 3 * 3 * 2 * 3)


def test_kernel_roofline_reports_serialised_kernels_and_the_overlapped_pass():
    N, M, B = 256, 64, 64
    L = N * N * M
    serial = [(0.020 * 320, 320), (0.018 * 320, 320), (0.017 * 320, 320), (0.0, 0)]   # 4 kinds, last unused
    over = ([(0.030 * 640, 640), (0.032 * 640, 640), (0.027 * 640, 640), (0.0, 0)], 20)
    r = bench.kernel_roofline(serial, N, M, B, 10, 6780.7, "measured", 2100.0, B * 12 * L, "f32", overlapped=over)
    assert r["kernel"] == "kf_fwd_xt"
    assert r["traffic"] == pytest.approx((33.603232 + 0.051648) * 1e6)
    assert r["avg_launch_ms"] == pytest.approx(0.020)
    assert [k["kernel"] for k in r["kernels_overlapped"]] == ["kf_fwd_xt", "kf_lines", "kf_inv_tx"]
    assert r["kernels_overlapped"][1]["avg_launch_ms"] == pytest.approx(0.032)
    assert "serialised" in r["timing"]
