"""The roofline arithmetic of bench.py (no GPU): achieved = algorithmic work
of the profiled iterations / their summed duration, frac = achieved / peak,
measured DRAM traffic only where one ncu capture describes every launch."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_fp64_bound_entry_uses_the_work_model_and_the_fp64_peak():
    work, unit, (bound, note), _ = bench.kernel_work_per_iteration("k_sdc_old", "bf16x3")
    assert unit == "flop" and bound == "alu" and note == "FP64 pipe"
    # 32 slices x 3 fields x ncoef(255) x 2 (M+1)(3M+1) flops with M = 4
    assert work == 32 * 3 * 32896 * 2 * 5 * 13
    e = bench.roofline_entry("k_sdc_old", 4, 0.84, "bf16x3", 2)
    assert e["bound"] == "alu" and e["peak"] == bench.ALU_PEAKS["fp64"][0] and e["unit"] == "TFLOP/s"
    assert e["peak_source"] == bench.ALU_PEAKS["fp64"][1]
    assert abs(e["achieved"] - work * 2 / 0.84e-3 / 1e12) < 1e-12
    assert abs(e["frac"] - e["achieved"] / e["peak"]) < 1e-15
    assert e["mean_launch_ms"] == pytest.approx(0.21)
    assert e["traffic"] == bench.NCU_TRAFFIC["k_sdc_old"][0]


def test_traffic_only_for_captured_uniform_kernels():
    assert bench.roofline_entry("k_grid_rhs", 160, 3.5, "bf16x3", 2)["traffic"] is None
    assert bench.roofline_entry("k_chain_node", 132, 3.8, "fp64", 2)["traffic"] is None   # FP64 build of the kernel
    assert bench.roofline_entry("k_chain_node", 132, 3.8, "bf16x3", 2)["traffic"] == \
        bench.NCU_TRAFFIC["k_chain_node"][0]
    for name, (_, _, src) in bench.NCU_TRAFFIC.items():
        assert os.path.exists(os.path.join(ROOT, src)), src


def test_hbm_entry_and_tensor_kernels_below_the_ridge():
    pk, _ = bench.peaks()
    e = bench.roofline_entry("k_grid_rhs", 160, 3.5, "bf16x3", 2)
    assert e["bound"] == "hbm" and e["peak"] == pk["hbm_gbs"] and e["unit"] == "GB/s"
    a = bench.roofline_entry("k_anal_bf16x3", 32, 1.8, "bf16x3", 2)
    assert a["bound"] == "hbm"                                 # 3xBF16 GEMMs at these widths sit below the ridge
    assert "below the ridge" in a["note"]


def test_cores_used_is_cpu_time_over_wall_time():
    assert bench.cores_used(10.0, 5.0) == 2
    assert bench.cores_used(0.2, 5.0) == 1
    assert bench.job_value(30.0, 2, 10) == pytest.approx(2 * 10 / 0.030)


def test_both_arms_print_the_same_metric_and_unit():
    """The reference arm and the GPU arm share METRIC/UNIT, so the two lines
    can be compared."""
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert src.count('"metric": METRIC') == 2
    assert '"unit": UNIT' in src


def test_proc_cpu_seconds_counts_this_process():
    import time
    t0 = bench.proc_cpu_seconds([os.getpid()])
    x = 0
    end = time.process_time() + 0.3
    while time.process_time() < end:
        x += 1
    assert bench.proc_cpu_seconds([os.getpid()]) - t0 > 0.1


def test_grid_work_is_split_between_the_long_and_short_row_kernels():
    """A row of nlon points takes the long-row kernel when its 10 padded
    transforms (nlon + nlon/16 + 1 complex entries) exceed 227 KB; the work
    model gives each kernel the rows it serves, so the two together carry the
    whole grid stage of the T1279/T639 workload."""
    assert bench.grid_long_rows(3840, 4) and bench.grid_long_rows(1536, 8)
    assert not bench.grid_long_rows(1920, 4) and not bench.grid_long_rows(768, 4)
    W = bench.Workload(1279, 639, 16, 5, 3)
    long_w = bench.kernel_work_per_iteration("k_grid_rhs_long", "bf16x3", W)[0]
    short_w = bench.kernel_work_per_iteration("k_grid_rhs", "bf16x3", W)[0]
    nfs, ncb, ncs = bench.rhs_states_per_iteration(W)
    (nlat_f, _), (nlat_c, _) = W.GRID_F, W.GRID_C
    assert long_w == nfs * bench.grid_rhs_bytes(1279, nlat_f, 1, 4)
    assert short_w == (ncb + ncs) * bench.grid_rhs_bytes(639, nlat_c, 1, 4)
    # at T255/T127 both levels take the short-row kernel
    assert bench.kernel_work_per_iteration("k_grid_rhs_long", "bf16x3")[0] == 0


def test_legendre_entry_count_of_one_direction():
    """(T+2)(T+3)/2 rows (m <= n <= T+1) times nlat/2 latitudes: 788,276,160
    entries at T1279 on 1920 latitudes, 3.15 GB as 3xBF16 images (4 bytes)."""
    W = bench.Workload(1279, 639, 16, 5, 3)
    entries = (W.TF + 2) * (W.TF + 3) // 2 * (W.GRID_F[0] // 2)
    assert entries == 788_276_160
    assert abs(entries * 4 / 1e9 - 3.153) < 1e-3
