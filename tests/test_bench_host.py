"""Host-side logic of bench.py on the CPU: the nvidia-smi clock summary
(median under load, throttle reasons), the lookup of a kernel's DRAM
traffic in the committed profile summaries (only while its source hash
matches), the roofline peak, and the JSON keys of the reference arm."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def sampler_with(lines):
    s = bench.ClockSampler(0)
    s.out = "\n".join(lines)
    return s


def test_clock_summary_median_under_load_and_reasons():
    rows = [
        "0, 1200, 2070, 150.00, 0x0, Not Active, Not Active, Not Active, Not Active",     # idle
        "0, 2070, 2070, 900.00, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1100.00, 0x4, Not Active, Not Active, Not Active, Active",        # power cap
        "0, 2070, 2070, 950.00, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    s = sampler_with(rows).summary(power_floor_w=500.0)
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    s_all = sampler_with(rows).summary()
    assert s_all["samples"] == 4 and s_all["sm_mhz"] == pytest.approx(2062.5)


def test_clock_summary_flags_thermal_slowdown_and_no_samples():
    rows = ["0, 1800, 2070, [N/A], 0x40, Active, Not Active, Active, Not Active"]
    s = sampler_with(rows).summary()
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    empty = sampler_with([]).summary()
    assert empty["sm_mhz"] is None and empty["reasons"] == ["no samples"]


def test_profile_traffic_only_for_matching_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k.md").write_text("# k\n\nkernel: merge_engine_kernel\nsource_sha: abc123\n"
                               "dram_bytes_per_output_element: 15.25\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda kernel="merge_engine_kernel": "abc123")
    value, path = bench.profile_traffic("merge_engine_kernel")
    assert value == 15.25 and path == os.path.join("profiles", "k.md")
    monkeypatch.setattr(bench, "kernel_source_sha", lambda kernel="merge_engine_kernel": "changed")
    assert bench.profile_traffic("merge_engine_kernel") == (None, None)
    assert bench.profile_traffic("other_kernel") == (None, None)


def test_committed_profile_names_a_source_hash():
    value, _ = bench.profile_traffic("merge_engine_kernel")
    sha = bench.kernel_source_sha("merge_engine_kernel")
    assert len(sha) == 16
    if value is not None:                        # the sources are those the counters were taken on
        assert 8.0 <= value <= 32.0


def test_peak_is_the_measured_copy_bandwidth():
    peak, kind = bench.measured_peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            assert (peak, kind) == (float(json.load(f)["hbm_gbs"]), "measured")
    else:
        assert (peak, kind) == (6800.0, "fallback")


def test_reference_arm_json_line_on_a_small_sample():
    """The reference arm on the host cores: one JSON line with the contract's
    keys (a 2^16-element workload here, so that it runs in seconds)."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                        "--log2n", "16"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_cpu_baselines_of_the_sort_and_batched_forms():
    s = bench.cpu_sort_baseline(log2n=16)
    assert s["value"] > 0 and s["cores"] == 1 and s["kind"] == "oracle" and s["equal_numpy_stable_sort"]
    b = bench.cpu_batched_baseline(pairs=64)
    assert b["value"] > 0 and b["cores"] == 1 and b["kind"] == "oracle"
    assert bench.guarded(lambda: 1 // 0) == {"error": "ZeroDivisionError: integer division or modulo by zero"}
    assert bench.guarded(lambda x: x + 1, 1) == 2


def test_cpu_baseline_of_the_lsm_form():
    d = bench.cpu_learned_baseline(log2_base=16, merges=3, log2_batch=10)
    assert d["value"] > 0 and d["cores"] == 1 and d["kind"] == "oracle" and "2^16" in d["sample"]
