"""Host-side logic of bench.py (CPU only): peak and work formulas, the DRAM
traffic table lookup, the roofline entry and the clock-log summary."""

import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PEAKS = {"hbm_gbs": 6788.3, "bf16_tflops": 1912.1, "bf16_tflops_sustained": 1717.8, "sm_max_mhz": 2070.0,
         "source": "measured"}


def test_peak_and_work_formulas(bench):
    assert bench.fp32_simt_peak_tflops(152, 2070.0) == pytest.approx(2 * 128 * 152 * 2070e6 / 1e12)
    assert bench.wprod_flops() == 2.0 * 256 ** 3 * 192


def test_traffic_table_follows_the_source_hash(bench, monkeypatch, tmp_path):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.md").write_text(
        "| kernel | source | source_sha16 | dram_bytes_per_launch |\n|---|---|---|---|\n"
        "| jacobi_svd | jacobi_block.cuh | 1234abcd5678ef90 | 31760000 |\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_src_hash", lambda fname: "1234abcd5678ef90")
    assert bench.ncu_traffic("jacobi_svd") == 31760000.0
    assert bench.ncu_traffic("no_such_kernel") is None
    monkeypatch.setattr(bench, "_src_hash", lambda fname: "0000000000000000")
    assert bench.ncu_traffic("jacobi_svd") is None       # source changed: no stale counters


def test_roofline_of_the_jacobi_kernel(bench):
    prof = {"jacobi_svd": (4, 40.0), "lift_forward": (8, 0.2)}     # (launches, total ms)
    jac = {"total_sweeps": 1000, "max_sweeps": 14}
    roof = bench._roofline(prof, PEAKS, 152, 2, True, jac)
    n, m = 256, 256
    per_sweep = (n - 1) * (n // 2) * m * 8 + 2 * m * n
    achieved = 1000 * per_sweep / 40e-3 / 1e12
    assert roof["kernel"] == "jacobi_svd" and roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert roof["achieved"] == pytest.approx(achieved)
    assert roof["frac"] == pytest.approx(achieved / bench.fp32_simt_peak_tflops(152, 2070.0))


def test_roofline_of_a_lifting_kernel(bench):
    prof = {"lift_forward": (2, 0.1)}
    roof = bench._roofline(prof, PEAKS, 152, 1, False)
    # two launches per step over A and B: 8 bytes per element, half per launch
    bytes_per_launch = 8.0 * 192 * (256 * 256 + 256 * 256) / 2
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["achieved"] == pytest.approx(bytes_per_launch / 50e-6 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 6788.3)


def test_clock_log_summary(bench, tmp_path):
    log = tmp_path / "clocks.csv"
    log.write_text("0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                   "0, 1965, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                   "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                   "garbage line\n")
    cs = bench.ClockSampler(0)
    cs.proc, cs.path = object(), str(log)
    summ = cs.summary()
    assert summ["sm_mhz"] == 2070.0 and summ["sm_max_mhz"] == 2070.0 and summ["samples"] == 3
    assert summ["reasons"] == ["sw_power_cap"]


def test_median_time_and_oracle_sample(bench):
    calls = []
    med, n = bench._median_time(lambda: calls.append(1), 5, 10.0)
    assert n == 5 and len(calls) == 5 and med >= 0.0
    # a budget already spent stops after the first call
    med, n = bench._median_time(lambda: __import__("time").sleep(0.01), 5, 0.0)
    assert n == 1
    # the w-svd sample is a whole number of tube groups and scales to the workload
    w = bench.WORKLOAD
    assert bench.SAMPLE_P % (1 << w["L"]) == 0 and bench.SAMPLE_P * bench.SAMPLE_SCALE == w["p"]
