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
    # the same config as the library's arm on this workload (its block count
    # is the library's default, one block per 2048 outputs)
    n = 1 << 16
    lengths = [(n, n)] * 4 + [(n, n >> 10)] * 4
    assert d["config"]["elements_per_step"] == sum(a + b for a, b in lengths)
    assert d["config"]["blocks_p"] == (2 * n) // 2048 and d["config"]["merges_per_step"] == 8


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


def _full_forms():
    per = {f"m{k}": 1.2345678 for k in range(8)}
    cpu = {"value": 7.1e8, "unit": "elems/s", "cores": 1, "kind": "oracle", "sample": "x" * 300, "seconds": 4.6}
    return {
        "merge_1m_p1024": {"workload": "w" * 200, "elements": 1572864, "us_per_merge": 27.1, "value": 5.8e10,
                           "gbs": 928.0, "fused": {"us_per_merge": 27.1}, "separate_launches": {"us_per_merge": 36.0},
                           "phases_us": {"search": 4.9, "barrier1": 1.5, "select": 2.5, "barrier2": 1.7,
                                         "merge": 11.0}},
        "batched": {"workload": "w" * 300, "value": 2.6e11, "ms": 2.97, "frac_of_hbm": 0.929, "config": {"tile": 2048},
                    "cpu_baseline": cpu, "bit_exact": True, "speedup_vs_plain": 468.7},
        "merge_sort": {"value": 1.17e10, "ms": 23.0, "frac_of_hbm": 0.79, "four_way_ms": 27.0,
                       "cpu_baseline": cpu, "bit_exact": True},
        "keys_only": {"uniform_full": {"ms": 1.24, "value": 4.3e11, "gbs": 3460.0, "frac_of_hbm": 0.51},
                      "uniform_1024": {"ms": 0.92, "value": 5.8e11, "gbs": 4660.0, "frac_of_hbm": 0.69}},
        "payload64": {"ms": 1.9, "value": 2.8e11, "gbs": 6780.0, "frac_of_hbm": 1.01, "workload": "w" * 80},
        "segmented_sort": {"ms": 40.0, "value": 1.9e10, "frac_of_hbm": 0.7, "bit_exact": True, "workload": "w" * 80},
        "partition_ablation": {"blocks": {"total_ms": 8.12, "per_merge_ms": per},
                               "equal_output": {"total_ms": 8.63, "per_merge_ms": per},
                               "equal_output_over_blocks": 1.063},
        "learned": {"plain": {"value": 3.99e11, "search_ms_mean": 0.055}, "learned": {"value": 4.0e11, "fallbacks": 0},
                    "search_speedup": 1.08, "search_speedup_pla_only": 1.07, "end_to_end_speedup": 1.004,
                    "bit_identical": True, "cpu_baseline": cpu},
    }


def test_compact_line_keeps_every_form_and_stays_short():
    line = {"metric": bench.METRIC, "value": 3.99e11, "unit": "elems/s", "n_gpus": 1, "steps": 200, "warmup": 5,
            "ms_per_step": 8.07, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic",
            "config": {"workload": bench.WORKLOAD_SHORT, "elements_per_step": 3222274048, "merges_per_step": 8,
                       "tile": 2048, "blocks_p": 262144, "threads": 128, "stages": "auto",
                       "split": "diagonal", "l2": "inputs > L2", "parallelism": "replicas x1", "phases": "overlap"},
            "forms": _full_forms(),
            "roofline": {"bound": "hbm", "kernel": "merge_engine_kernel", "achieved": 6760.0065, "peak": 6703.8,
                         "unit": "GB/s", "frac": 1.0083, "peak_kind": "measured hbm_gbs (copy)",
                         "traffic": 6162599116.8, "traffic_source": "profiles/merge_engine_kernel_large_merge.md",
                         "algorithmic_bytes_per_launch": 6444548096.0, "search_share": 0.0385,
                         "plan_share": 0.0145, "frac_of_nominal": 0.845, "frac_alone": 1.0102, "step_frac": 0.95},
            "cpu_baseline": {"value": 7.0e8, "unit": "elems/s", "cores": 1, "kind": "oracle", "sample": "y" * 200,
                             "seconds": 4.6, "e2e_outputs_equal_oracle": True,
                             "paper_parallel": {"value": 9.6e9, "cores": 16, "sample": "z" * 100}},
            "e2e": {"value": 1.6e10, "unit": "elems/s", "h2d_bytes_per_step": 25778192384,
                    "d2h_bytes_per_step": 25778192384, "steps": 3, "path": "p" * 200},
            "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 12},
            "gpu_launches": 4800}
    c = bench.compact_line(line, 6703.8)
    s = json.dumps(c, separators=(",", ":"))
    assert len(s) < 2400, len(s)           # whole inside a log cut to its last 3000 characters
    for form in ("merge_1m_p1024", "batched", "merge_sort", "keys_only", "learned", "partition_ablation",
                 "payload64", "segmented_sort"):
        assert form in c["forms"]
    assert c["forms"]["merge_1m_p1024"]["us"] == 27.1
    assert c["forms"]["merge_1m_p1024"]["phases_us"]["merge"] == 11.0
    assert c["forms"]["batched"]["frac_of_hbm"] == 0.929 and c["forms"]["batched"]["cpu"] == 7.1e8
    assert c["forms"]["keys_only"]["uniform_full"]["frac_of_hbm"] == 0.51
    assert c["forms"]["learned"]["search_speedup_pla_only"] == 1.07
    for key in ("value", "ms_per_step", "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches", "config"):
        assert key in c
    assert c["e2e"]["h2d_bytes_per_step"] == 25778192384
    assert c["roofline"]["frac"] == 1.0083 and c["roofline"]["bound"] == "hbm"
    # a failed form keeps a short error record
    forms = _full_forms()
    forms["batched"] = {"error": "RuntimeError: " + "e" * 500}
    c2 = bench.compact_forms(forms, 6703.8)
    assert c2["batched"]["error"].startswith("RuntimeError") and len(c2["batched"]["error"]) <= 160
