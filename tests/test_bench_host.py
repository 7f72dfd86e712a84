"""Host logic of bench.py on the CPU: the clock sampler against a fake nvidia-smi (the
samples inside the timed region and the two that bracket it are kept, throttle reasons are
collected, every wait is bounded), and the roofline denominators read from the measured
peaks file."""
import os
import sys
import time

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _fake_smi(rows, period_s=0.03, delay_s=0.0):
    """A stand-in for nvidia-smi --query-gpu ... -lms: prints one CSV row every period_s."""
    script = ("import sys, time\n"
              f"time.sleep({delay_s})\n"
              f"rows = {rows!r}\n"
              "i = 0\n"
              "while True:\n"
              "    print(rows[min(i, len(rows) - 1)], flush=True)\n"
              "    i += 1\n"
              f"    time.sleep({period_s})\n")
    return [sys.executable, "-c", script]


NORMAL = "2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
CAPPED = "1890, 2070, 1395.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
THERMAL = "1500, 2070, 1100.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active"


def test_samples_inside_and_around_the_region():
    with bench.Clocks(0, period_ms=30, cmd=_fake_smi([NORMAL], delay_s=0.2)) as clk:
        assert clk.lines, "the first sample is awaited before the region opens"
        time.sleep(0.2)
    s = clk.summary()
    assert s["in_region"] >= 3 and s["samples"] >= s["in_region"] + 1
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == []


def test_throttle_reasons_are_collected():
    rows = [NORMAL] * 3 + [CAPPED] * 3 + [THERMAL] * 100
    with bench.Clocks(0, period_ms=30, cmd=_fake_smi(rows)) as clk:
        time.sleep(0.4)
    s = clk.summary()
    assert "sw_power_cap" in s["reasons"] and "hw_thermal_slowdown" in s["reasons"]
    assert s["sm_mhz"] < 2070.0


def test_short_region_keeps_the_bracketing_samples():
    # a region shorter than the sampling period still has the sample before and after it
    with bench.Clocks(0, period_ms=200, cmd=_fake_smi([NORMAL], period_s=0.2)) as clk:
        pass
    s = clk.summary()
    assert s["samples"] >= 2 and s["sm_mhz"] == 2070.0


def test_missing_or_silent_sampler_does_not_hang():
    t = time.monotonic()
    with bench.Clocks(0, cmd=["/nonexistent/nvidia-smi"]) as clk:
        pass
    assert clk.summary()["samples"] == 0
    with bench.Clocks(0, cmd=[sys.executable, "-c", "pass"], start_timeout_s=1.0) as clk:
        pass
    assert clk.summary()["samples"] == 0
    assert time.monotonic() - t < 10.0


def test_peaks_come_from_the_measured_file_when_present():
    p = bench.peaks()
    assert set(p) >= {"hbm_gbs", "bf16_tflops", "bf16_tflops_sustained", "src"}
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert p["src"] == "measured" and p["hbm_gbs"] > 1000 and p["bf16_tflops"] > 100
    else:
        assert p["src"] == "fallback"


def test_forward_error_of_column_major_factors_ignores_the_upper_input():
    import numpy as np
    import paper_2601_08082_gb300.hrp as hrp
    rng = np.random.default_rng(3)
    n = 9
    L = np.tril(rng.standard_normal((n, n))) + 3 * np.eye(n)
    D = np.tril(rng.standard_normal((n, n))) * 1e-3
    M1 = L + np.triu(rng.standard_normal((n, n)), 1)        # strict upper: untouched input
    M2 = (L + D) + np.triu(rng.standard_normal((n, n)), 1)  # different garbage there
    fe = bench.forward_error_colmajor(hrp.colmajor(M2), hrp.colmajor(M1))
    assert abs(fe - np.linalg.norm(D) / np.linalg.norm(L)) <= 1e-12


def test_lpt_partition_covers_every_system_once_and_balances_the_work():
    import numpy as np
    rng = np.random.default_rng(7)
    n = rng.integers(64, 2049, size=2048)
    costs = [float(x) ** 3 for x in n]
    for world in (1, 2, 4, 8):
        parts = bench.lpt_partition(costs, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # Graham: LPT <= 4/3 OPT, and OPT >= max(mean load, largest item)
        opt_lb = max(sum(costs) / world, max(costs))
        assert max(loads) <= 4.0 / 3.0 * opt_lb
        assert max(loads) - min(loads) <= max(costs)      # list scheduling: within one item
    assert bench.lpt_partition([5.0, 5.0, 5.0], 2) == [[0, 2], [1]]   # ties by index, then rank
    assert bench.lpt_partition([], 3) == [[], [], []]


@pytest.mark.parametrize("warmup", [0, 1, 3, 5, 7])
def test_accuracy_entries_name_the_matrix_each_step_factored(warmup):
    # step s factors copies[s] = A0[s % 3]; the accuracy entry of a step must carry that
    # matrix's rho whatever the number of warm-up steps
    nsteps = warmup + 24
    seen = bench.accuracy_steps(warmup, nsteps, 3)
    assert [s for s, _ in seen] == [warmup, warmup + 1, warmup + 2]
    assert all(k == s % 3 for s, k in seen)
    assert sorted(k for _, k in seen) == [0, 1, 2]
    assert bench.accuracy_steps(warmup, warmup + 1, 3) == [(warmup, warmup % 3)]


def test_leaf_traffic_is_keyed_to_the_kernel_code(tmp_path):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n\ncudaError_t launch_k() { return 0; }\n")
    a = bench.device_code_sha1(str(src), "cudaError_t launch_k(")
    src.write_text("__global__ void k() {}\n\ncudaError_t launch_k() { return 1; /* host change */ }\n")
    assert bench.device_code_sha1(str(src), "cudaError_t launch_k(") == a
    src.write_text("__global__ void k() { int x; }\n\ncudaError_t launch_k() { return 1; }\n")
    assert bench.device_code_sha1(str(src), "cudaError_t launch_k(") != a


@pytest.mark.parametrize("n", [1, 127, 128, 129, 300, 1000])
def test_host_lower_bytes_counts_the_transferred_entries(n):
    # hrp_potrf_host transfers entry (i, j) when i >= 128 floor(j / 128)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    assert bench.host_lower_bytes(n) == 8 * int(np.count_nonzero(i >= 128 * (j // 128)))


def test_paired_ratio_ci_brackets_the_ratio():
    rng = np.random.default_rng(3)
    b = rng.uniform(10, 20, 40)
    a = 0.8 * b * rng.uniform(0.95, 1.05, 40)
    r, lo, hi = bench.paired_ratio_ci(a, b)
    assert abs(r - a.mean() / b.mean()) < 1e-15
    assert lo <= r <= hi and hi - lo < 0.05
    assert bench.paired_ratio_ci(b, b)[1:] == (1.0, 1.0)     # identical pairs: no spread


def test_cpu_dense_sample_times_the_oracle_on_a_bounded_prefix():
    from synth import rbf_spd, seed_for
    mats = [rbf_spd(n, seed_for(3, 1 + i)) for i, n in enumerate([64, 96, 80])]
    out = bench.cpu_dense_sample(mats, budget_s=0.0)       # stops after the first system
    assert out["kind"] == "oracle" and out["unit"] == "TFLOP/s" and out["cores"] >= 1
    assert out["value"] > 0 and "first 1 of the batch's systems" in out["sample"]
    out = bench.cpu_dense_sample(mats, budget_s=1e9)       # all of them
    assert "first 3 of the batch's systems" in out["sample"]
