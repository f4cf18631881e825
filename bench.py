"""Benchmark of the GB300 stable parallel merge.

Workload (the large single stable merge): n = m = 2**28 int32 keys with
int32 payloads in four seeded key distributions (uniform over the full int32
range, uniform in [0, 1024), all keys equal, Zipf s = 1.2 over 2**20 values),
plus the skewed lengths n = 2**28, m = 2**18 of the same four distributions:
eight merges per step, both inputs pre-sorted.  Metric: merged key+value
elements per second (n + m per merge), whole job.

One step = for each of the eight inputs, Steps 1-2 (cross-rank search
kernel), Steps 3-4 selection (planning kernel: one tile record per
subproblem) and Steps 3-4 merges (persistent staged tile-merge kernel),
through the C ABI phase calls tm_cross_ranks, tm_plan_subproblems and
tm_merge_tiles: the kernels tm_merge launches, with CUDA events between
them.
Inputs are resident in HBM; every merge reads 2-4 GB, far above the 129 MB
L2, so no L2 flush is needed between iterations.

Prints ONE JSON line on rank 0.  Under torchrun each rank runs an
independent replica on its own GPU (the merge has no exchange step), and
`value` counts the elements of all ranks over the slowest rank's time.

--impl reference times the CPU oracle (the plain two-pointer stable merge
of oracle/, single thread) on the same workload and prints the same line.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np
import torch

METRIC = "merged key+value elems/s and % of HBM peak, plain vs batched/learned, bit-exact"
WORKLOAD = ("stable merge, int32 keys + int32 payloads: n=m=2^28 x {uniform_full, uniform_1024, "
            "all_equal, zipf_1.2}, plus skewed n=2^28, m=2^18 x the same four; pre-sorted")
WORKLOAD_SHORT = "stable merge i32 keys+payloads: n=m=2^28 x 4 dists + skewed n=2^28, m=2^18 x 4"
UNIT = "elems/s"
NOMINAL_HBM_GBS = 8000.0


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Source files each profiled kernel is compiled from; a profile's counters
# stand only while these files are unchanged.
KERNEL_SOURCES = {
    "merge_engine_kernel": ["tm_engine.cuh", "tm_engine_launch.cuh", "tm_engine_i32.cu", "tm_engine_u32.cu",
                            "tm_engine_u64.cu", "tm_engine_f32.cu", "tm_engine_i32_v64.cu", "tm_engine_u32_v64.cu",
                            "tm_engine_u64_v64.cu", "tm_engine_f32_v64.cu", "tm_common.cuh", "tm_host.h"],
}


def kernel_source_sha(kernel: str = "merge_engine_kernel") -> str:
    h = hashlib.sha256()
    names = KERNEL_SOURCES.get(kernel)
    files = ([os.path.join(ROOT, "paper_1202_6575_gb300", "csrc", f) for f in names] if names else
             sorted(glob.glob(os.path.join(ROOT, "paper_1202_6575_gb300", "csrc", "*"))))
    for f in files:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_traffic(kernel: str):
    """DRAM bytes per output element of `kernel` from the committed ncu
    summary, if it was taken on the current kernel sources."""
    sha = kernel_source_sha(kernel)
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        txt = open(path).read()
        m_k = re.search(r"^kernel:\s*(\S+)", txt, re.M)
        m_s = re.search(r"^source_sha:\s*(\S+)", txt, re.M)
        m_b = re.search(r"^dram_bytes_per_output_element:\s*([0-9.]+)", txt, re.M)
        if m_k and m_s and m_b and m_k.group(1) == kernel and m_s.group(1) == sha:
            return float(m_b.group(1)), os.path.relpath(path, ROOT)
    return None, None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 50):
        self.gpu = gpu_index
        self.proc = None
        self.interval_ms = interval_ms

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 f"-lms={self.interval_ms}"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self, power_floor_w: float = 0.0):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append({"sm": float(parts[1]), "max": float(parts[2]),
                             "power": float(parts[3]) if parts[3] not in ("[N/A]", "N/A") else 0.0,
                             "hw": parts[5], "hw_thermal": parts[6], "sw_thermal": parts[7],
                             "sw_power": parts[8]})
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        load = [r for r in rows if r["power"] >= power_floor_w] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hw_thermal", "hw_thermal_slowdown"),
                              ("sw_thermal", "sw_thermal_slowdown"), ("sw_power", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median([r["sm"] for r in load])),
                "sm_max_mhz": max(r["max"] for r in rows), "reasons": sorted(reasons),
                "samples": len(load)}


def max_over_ranks(ms: float, device) -> float:
    """The slowest rank's time (all ranks get it)."""
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Units all ranks processed divided by the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1e3)


def make_inputs(device, log2n=28, dists=None, skewed_too=True):
    from paper_1202_6575_gb300 import workloads as W
    items = []
    for skewed in ((False, True) if skewed_too else (False,)):
        for dist in (dists or W.DIST_NAMES):
            A, Av, B, Bv = W.large_merge(dist, skewed, device, log2n=log2n, log2m_skewed=log2n - 10)
            items.append({"name": f"{dist}{'_skewed' if skewed else ''}", "A": A, "Av": Av, "B": B, "Bv": Bv})
    return items


def headline_config(args, world: int, lengths: list, p=None) -> dict:
    """The large-merge workload's config, the same on both arms; lengths:
    (n, m) of every merge of a step; p: the first merge's block count (the
    library's default, one block per tile of outputs, when not given)."""
    n0, m0 = lengths[0]
    tile = args.tile or 2048
    return {"workload": WORKLOAD_SHORT, "elements_per_step": sum(n + m for n, m in lengths),
            "merges_per_step": len(lengths), "tile": tile,
            "blocks_p": p if p is not None else -(-(n0 + m0) // tile),
            "threads": args.threads or 128, "stages": args.stages or "auto",
            "split": {0: "diagonal", 1: "blocks", 2: "diagonal"}[args.split],
            "l2": "inputs > L2", "parallelism": f"replicas x{world}",
            "phases": "serial" if args.serial else "overlap"}


def run_reference(args, rank, world):
    """The CPU oracle on the host cores (rank 0 only; other ranks exit).

    Each step merges a bounded sample of the workload: step k takes merge
    k mod 8 of the workload restricted to the prefixes A[:a], B[:b] with
    a : b = n : m, sized so that warmup + steps finish in about 90 s of CPU
    time.  The two-pointer merge costs the same per element at any length,
    so the rate carries over to the full workload."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    gen_dev = "cuda" if torch.cuda.is_available() else "cpu"
    items = make_inputs(gen_dev, args.log2n, args.dists, not args.no_skewed)
    hosts = [(it["A"].cpu().numpy(), it["Av"].cpu().numpy().view(np.uint32),
              it["B"].cpu().numpy(), it["Bv"].cpu().numpy().view(np.uint32)) for it in items]
    del items
    # calibrate the single-thread rate on a 2**24-element prefix
    A, Av, B, Bv = hosts[0]
    t0 = time.perf_counter()
    oracle.merge_two_pointer(A[:1 << 23], Av[:1 << 23], B[:1 << 23], Bv[:1 << 23])
    rate = (1 << 24) / (time.perf_counter() - t0)
    total_steps = args.steps + args.warmup
    per_step = int(min(max(rate * 90.0 / total_steps, 1 << 20), len(A) + len(B)))

    def step(k):
        A, Av, B, Bv = hosts[k % len(hosts)]
        n, m = len(A), len(B)
        a = int(round(per_step * n / (n + m)))
        b = min(m, per_step - a)
        oracle.merge_two_pointer(A[:a], Av[:a], B[:b], Bv[:b])
        return a + b

    for k in range(args.warmup):
        step(k)
    elems = 0
    t0 = time.perf_counter()
    for k in range(args.steps):
        elems += step(args.warmup + k)
    dt = time.perf_counter() - t0
    value = elems / dt
    sample = (f"per step, prefixes of one of the eight merges (round robin) totalling {per_step} elements; "
              f"single-thread two-pointer oracle (oracle/tm_oracle.c)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic", "config": headline_config(args, world, [(len(h[0]), len(h[2])) for h in hosts]),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(items):
    """Times the oracle, as it stands, on one merge of each input (host
    copies), and compares its results with the end-to-end run's outputs."""
    import oracle
    oracle.build()
    hosts = [(it["hA"], it["hAv"].view(np.uint32), it["hB"], it["hBv"].view(np.uint32)) for it in items]
    elems = sum(len(h[0]) + len(h[2]) for h in hosts)
    same = True
    dt = 0.0
    for it, (A, Av, B, Bv) in zip(items, hosts):
        t0 = time.perf_counter()
        K, V = oracle.merge_two_pointer(A, Av, B, Bv)
        dt += time.perf_counter() - t0
        if "hC" in it:
            same = same and np.array_equal(it["hC"].numpy(), K.view(np.int32)) and \
                np.array_equal(it["hCv"].numpy().view(np.uint32), V)
    # second baseline: the paper's algorithm on every host core (one thread
    # per processing element, p = cores), same merges
    cores = os.cpu_count() or 1
    dtp = 0.0
    same_par = True
    for it, (A, Av, B, Bv) in zip(items, hosts):
        t0 = time.perf_counter()
        Kp, Vp, _, _ = oracle.paper_merge_parallel(A, Av, B, Bv, cores, cores)
        dtp += time.perf_counter() - t0
        if "hC" in it:                                  # the e2e outputs, equal to the oracle's above
            same_par = same_par and np.array_equal(it["hC"].numpy(), Kp.view(np.int32)) and \
                np.array_equal(it["hCv"].numpy().view(np.uint32), Vp)
        del Kp, Vp
    return {"value": elems / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "each of the eight merges once (the full workload, one pass), single-thread "
                      "two-pointer merge of oracle/tm_oracle.c", "seconds": dt,
            "e2e_outputs_equal_oracle": bool(same),
            "paper_parallel": {"value": elems / dtp, "unit": UNIT, "cores": cores, "p": cores,
                               "kind": "paper's algorithm on POSIX threads (oracle/paper_parallel.c)",
                               "sample": "the same eight merges once", "seconds": dtp,
                               "outputs_equal_e2e": bool(same_par)}}


def cpu_sort_baseline(log2n: int = 22):
    """The oracle's stable merge sort (bottom-up from runs of one element,
    oracle/tm_oracle.c), as it stands, on one host core, over a bounded
    sample of the sort workload: 2**log2n u64 keys of the same distribution
    (uniform in [0, 2**24)) with index payloads, sorted once; checked
    against numpy's stable sort."""
    import oracle
    from paper_1202_6575_gb300 import workloads as W
    n = 1 << log2n
    keys, vals = W.sort_input("cpu", n=n)
    hk, hv = keys.numpy().view(np.uint64), vals.numpy().view(np.uint32)
    t0 = time.perf_counter()
    k, v = oracle.merge_sort(hk, hv, run=1)
    dt = time.perf_counter() - t0
    order = np.argsort(hk, kind="stable")
    return {"value": n / dt, "unit": "sorted elems/s", "cores": 1, "kind": "oracle",
            "sample": f"2^{log2n} keys of the same distribution, sorted once (bottom-up merge sort)",
            "seconds": dt, "equal_numpy_stable_sort": bool(np.array_equal(k, hk[order]) and
                                                           np.array_equal(v, hv[order]))}


def cpu_batched_baseline(pairs: int = 2048):
    """The oracle's independent two-pointer merges, as they stand, on one
    host core, over a bounded sample of the batched workload: `pairs` pairs
    of the same length distribution (log-uniform in [1, 2**16] per side, u64
    keys), merged once."""
    import oracle
    from paper_1202_6575_gb300 import workloads as W
    a_off, A, Av, b_off, B, Bv = W.batched_pairs("cpu", pairs=pairs)
    total = A.numel() + B.numel()
    args = (a_off.numpy(), A.numpy().view(np.uint64), Av.numpy().view(np.uint32),
            b_off.numpy(), B.numpy().view(np.uint64), Bv.numpy().view(np.uint32))
    t0 = time.perf_counter()
    oracle.merge_batched(*args)
    dt = time.perf_counter() - t0
    return {"value": total / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{pairs} pairs of the same length distribution ({total:,} elements), merged once",
            "seconds": dt}


def cpu_learned_baseline(log2_base: int = 24, merges: int = 16, log2_batch: int = 20):
    """The oracle's two-pointer merge, as it stands, on one host core, over a
    bounded sample of the LSM workload: a 2**log2_base base of the same
    mixture merged `merges` times with its sorted 2**log2_batch batches
    (base' = merge(base, batch), the base on the A side).  The oracle needs
    no model: its rate per merged element is that of any plain merge."""
    import oracle
    from paper_1202_6575_gb300 import workloads as W
    N0, m = 1 << log2_base, 1 << log2_batch
    X, Xv = W.lsm_base("cpu", n=N0)
    base, base_v = X.numpy(), Xv.numpy().view(np.uint32)
    elems, dt = 0, 0.0
    for k in range(merges):
        B, Bv = W.lsm_batch(k, "cpu", size=m, base_n=N0)
        t0 = time.perf_counter()
        base, base_v = oracle.merge_two_pointer(base, base_v, B.numpy(), Bv.numpy().view(np.uint32))
        dt += time.perf_counter() - t0
        elems += len(base)
    return {"value": elems / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"base 2^{log2_base} of the same mixture merged {merges} times with sorted 2^{log2_batch} "
                      "batches (two-pointer merge)", "seconds": dt}


def _r(x, digits=4):
    """x rounded to `digits` significant digits (None and non-numbers pass)."""
    if isinstance(x, (bool, int)) or not isinstance(x, float):   # counts stay exact
        return x
    if x == 0 or not np.isfinite(x):
        return float(x)
    return float(f"{x:.{digits}g}")


def compact_forms(forms: dict, peak_gbs: float) -> dict:
    """The figures of every side form that the one-line result keeps: value,
    time, fraction of the measured copy bandwidth, the CPU baseline's value
    and the exactness flag.  Everything else (per-merge times, ablation
    detail, configurations) goes to the detail line printed before it."""
    if not forms:
        return forms
    out = {}
    g = lambda d, k: (d or {}).get(k) if isinstance(d, dict) else None
    f = forms.get("merge_1m_p1024")
    if isinstance(f, dict) and "error" not in f:
        out["merge_1m_p1024"] = {"value": _r(f.get("value")), "us": _r(f.get("us_per_merge")),
                                 "frac_of_hbm": _r(g(f, "gbs") / peak_gbs if g(f, "gbs") else None),
                                 "separate_us": _r(g(g(f, "separate_launches"), "us_per_merge")),
                                 "phases_us": {k: _r(v, 3) for k, v in (g(f, "phases_us") or {}).items()} or None}
    f = forms.get("batched")
    if isinstance(f, dict) and "error" not in f:
        out["batched"] = {"value": _r(f.get("value")), "ms": _r(f.get("ms")), "frac_of_hbm": _r(f.get("frac_of_hbm")),
                          "cpu": _r(g(g(f, "cpu_baseline"), "value")), "bit_exact": f.get("bit_exact")}
    f = forms.get("merge_sort")
    if isinstance(f, dict) and "error" not in f:
        out["merge_sort"] = {"value": _r(f.get("value")), "ms": _r(f.get("ms")),
                             "frac_of_hbm": _r(f.get("frac_of_hbm")), "four_way_ms": _r(f.get("four_way_ms")),
                             "cpu": _r(g(g(f, "cpu_baseline"), "value")), "bit_exact": f.get("bit_exact")}
    f = forms.get("keys_only")
    if isinstance(f, dict) and "error" not in f:
        out["keys_only"] = {d: {"value": _r(g(f[d], "value")), "ms": _r(g(f[d], "ms")),
                                "frac_of_hbm": _r(g(f[d], "frac_of_hbm"))}
                            for d in ("uniform_full", "uniform_1024") if d in f}
    f = forms.get("learned")
    if isinstance(f, dict) and "error" not in f:
        out["learned"] = {"value": _r(g(g(f, "learned"), "value")), "plain_value": _r(g(g(f, "plain"), "value")),
                          "e2e_speedup": _r(f.get("end_to_end_speedup")),
                          "search_speedup": _r(f.get("search_speedup")),
                          "search_speedup_pla_only": _r(f.get("search_speedup_pla_only")),
                          "e2e_speedup_pla_only": _r(f.get("end_to_end_speedup_pla_only")),
                          "mlp_vs_pla_search": _r(f.get("mlp_vs_pla_search")),
                          "fallbacks": g(g(f, "learned"), "fallbacks"), "bit_identical": f.get("bit_identical"),
                          "cpu": _r(g(g(f, "cpu_baseline"), "value"))}
    f = forms.get("payload64")
    if isinstance(f, dict) and "error" not in f:
        out["payload64"] = {"value": _r(f.get("value")), "ms": _r(f.get("ms")), "frac_of_hbm": _r(f.get("frac_of_hbm"))}
    f = forms.get("segmented_sort")
    if isinstance(f, dict) and "error" not in f:
        out["segmented_sort"] = {"value": _r(f.get("value")), "ms": _r(f.get("ms")),
                                 "frac_of_hbm": _r(f.get("frac_of_hbm")), "bit_exact": f.get("bit_exact")}
    f = forms.get("partition_ablation")
    if isinstance(f, dict) and "error" not in f:
        out["partition_ablation"] = {"equal_output_over_blocks": _r(f.get("equal_output_over_blocks"))}
    for k, f in forms.items():                         # a form that failed keeps its one-line error
        if isinstance(f, dict) and "error" in f:
            out[k] = {"error": str(f["error"])[:160]}
    return out


def compact_line(line: dict, peak_gbs: float) -> dict:
    """The result line with its long parts shortened: the side forms reduced
    by compact_forms, the baselines' descriptions cut, numbers rounded."""
    out = dict(line)
    out["forms"] = compact_forms(line.get("forms"), peak_gbs)
    cpu = line.get("cpu_baseline")
    if isinstance(cpu, dict):
        c = {k: _r(cpu.get(k)) for k in ("value", "unit", "cores", "kind")}
        c["sample"] = "8 merges once, two-pointer oracle"
        c["e2e_outputs_equal_oracle"] = cpu.get("e2e_outputs_equal_oracle")
        pp = cpu.get("paper_parallel")
        if isinstance(pp, dict):
            c["paper_parallel"] = {"value": _r(pp.get("value")), "cores": pp.get("cores")}
        out["cpu_baseline"] = c
    e2e = line.get("e2e")
    if isinstance(e2e, dict):
        out["e2e"] = {k: _r(v) for k, v in e2e.items() if k != "path"}
    rl = line.get("roofline")
    if isinstance(rl, dict):
        out["roofline"] = {k: _r(v, 5) for k, v in rl.items() if k not in ("traffic_source", "peak_kind")}
        out["roofline"]["peak_kind"] = "measured copy" if "measured" in str(rl.get("peak_kind")) else "fallback"
    return out


def guarded(fn, *args, **kwargs):
    """fn's result, or its error as a one-line record (a report extra must
    not lose the benchmark line)."""
    try:
        return fn(*args, **kwargs)
    except Exception as e:                              # noqa: BLE001
        return {"error": f"{type(e).__name__}: {e}"}



# Elements per initial sorted run of tm_merge_sort (one CTA's radix sort);
# the merge rounds double it.
SORT_RUN = 4096

def side_stream(dev):
    """A new stream whose work starts after everything already issued on the
    current stream.  The inputs are generated there; without the wait, a
    kernel on the new stream can read them half written, or overwrite a
    block the caching allocator has just handed back while a kernel on the
    current stream still reads it."""
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    return s

def bench_small_merge(dev, steps: int = 200):
    """The 1M merge: A n = 2**20, B m = 2**19 u32 keys in [0, 2**16), p = 1024
    blocks per input; one tm_merge captured in a CUDA graph and replayed (a
    merge of 25 MB is launch-latency bound).  L2 is flushed (a 256 MB write)
    before every timed replay; each replay is timed alone with CUDA events
    and the median reported."""
    from paper_1202_6575_gb300 import tm, workloads as W
    A, Av, B, Bv = W.single_merge_1m(dev)
    n, m = A.numel(), B.numel()
    C = torch.empty(n + m, dtype=torch.int32, device=dev)
    Cv = torch.empty(n + m, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    s = side_stream(dev)
    out = {"workload": "A 2^20 + B 2^19 u32 keys in [0, 2^16), u32 payloads, p = 1024; one CUDA graph replay "
                       "per merge", "elements": n + m, "unit": UNIT, "l2": "flushed before every replay"}
    ref = None
    graphs = []                          # kept alive: destroying a graph during a capture invalidates it
    for name, cfg in (("fused", {"p": 1024}), ("separate_launches", {"p": 1024, "unfused": 1})):
        ws = tm.new_workspace(tm.tm_merge_workspace_size(n, m, cfg), dev)
        tm.tm_merge("u32", A, Av, B, Bv, C, Cv, ws, cfg=cfg, stream=s)
        s.synchronize()
        g = tm.Graph(s)
        graphs.append(g)
        with g:
            tm.tm_merge("u32", A, Av, B, Bv, C, Cv, ws, cfg=cfg, stream=s)
        for _ in range(10):
            g.launch()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        with torch.cuda.stream(s):
            for i, (e0, e1) in enumerate(evs):
                flush.fill_(i & 255)
                e0.record(s)
                g.launch()
                e1.record(s)
        s.synchronize()
        us = float(np.median([e0.elapsed_time(e1) * 1e3 for e0, e1 in evs]))
        assert tm.tm_read_status(ws, stream=s) == 0
        if ref is None:
            ref = (C.clone(), Cv.clone())
        else:
            assert torch.equal(ref[0], C) and torch.equal(ref[1], Cv)
        out[name] = {"us_per_merge": us, "value": (n + m) / (us / 1e6), "gbs": (n + m) * 16 / (us / 1e6) / 1e9,
                     "graph": "memset, fused search + merge kernel" if name == "fused" else
                              "memset, search, plan, memset, merge"}
    out.update({"us_per_merge": out["fused"]["us_per_merge"], "value": out["fused"]["value"],
                "gbs": out["fused"]["gbs"]})
    # where the fused launch spends its time: per-CTA %globaltimer stamps
    # (tm_config.trace), L2 flushed before each of 20 traced calls, median
    cfg = {"p": 1024, "trace": 1}
    ws = tm.new_workspace(tm.tm_merge_workspace_size(n, m, cfg), dev)
    phases = []
    for i in range(23):
        with torch.cuda.stream(s):                     # the flush ends before the traced merge starts
            flush.fill_(i & 255)
        tm.tm_merge("u32", A, Av, B, Bv, C, Cv, ws, cfg=cfg, stream=s)
        ph = tm.tm_merge_phase_times(ws, n, m, cfg, stream=s)
        if i >= 3:
            phases.append(ph)
    assert tm.tm_read_status(ws, stream=s) == 0
    assert torch.equal(ref[0], C) and torch.equal(ref[1], Cv)
    out["phases_us"] = {k: float(np.median([ph[k] for ph in phases])) for k in tm.PHASES}
    # the last traced call per CTA: when each CTA passed the barrier, landed
    # its first tile and finished, against its tile count (the merge phase
    # ends with the last CTA)
    tr = tm.tm_merge_trace(ws, n, m, cfg, stream=s).astype(np.int64)
    t0 = tr[:, 0].min()
    rel = lambda col: (tr[:, col] - t0) / 1e3
    done, tiles = rel(5), tr[:, 7]
    out["per_cta"] = {
        "ctas": int(tr.shape[0]),
        "barrier_passed_us": {"median": float(np.median(rel(2))), "max": float(rel(2).max())},
        "first_tile_us": {"median": float(np.median(rel(6))), "max": float(rel(6).max())},
        "merges_done_us": {"median": float(np.median(done)), "p90": float(np.percentile(done, 90)),
                           "max": float(done.max())},
        "tiles": {int(k): {"ctas": int((tiles == k).sum()), "done_median_us": float(np.median(done[tiles == k]))}
                  for k in np.unique(tiles)}}
    return out


def bench_partition(dev, reps: int = 5):
    """Ablation: the eight large merges partitioned by the paper's blocks
    (cross ranks of block starts, the five cases; the default) and by equal
    output ranges (one co-rank search per 2048 outputs, prior work the paper
    discusses), each through tm_merge; median of `reps` calls per merge."""
    from paper_1202_6575_gb300 import tm
    items = make_inputs(dev, 28, None, True)
    out = {"workload": "the eight large merges (n = m = 2^28 and n = 2^28, m = 2^18 int32 keys + payloads)",
           "unit": "ms"}
    for name, cfg in (("blocks", {"partition": 0, "unfused": 1}), ("equal_output", {"partition": 1})):
        per = {}
        for it in items:
            A, Av, B, Bv = it["A"], it["Av"], it["B"], it["Bv"]
            n, m = A.numel(), B.numel()
            C = torch.empty(n + m, dtype=torch.int32, device=dev)
            Cv = torch.empty(n + m, dtype=torch.int32, device=dev)
            ws = tm.new_workspace(tm.tm_merge_workspace_size(n, m, cfg), dev)
            tm.tm_merge("i32", A, Av, B, Bv, C, Cv, ws, cfg=cfg)
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                tm.tm_merge("i32", A, Av, B, Bv, C, Cv, ws, cfg=cfg)
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            assert tm.tm_read_status(ws) == 0
            per[it["name"]] = float(np.median(ts))
            del C, Cv, ws
        out[name] = {"total_ms": sum(per.values()), "per_merge_ms": per}
    out["equal_output_over_blocks"] = out["equal_output"]["total_ms"] / out["blocks"]["total_ms"]
    for it in items:
        it.clear()
    torch.cuda.empty_cache()
    return out


def bench_keys_only(dev, steps: int = 20):
    """Keys-only merges (payload pointers NULL): n = m = 2**28 int32 keys,
    uniform in [0, 1024) and uniform over int32; 8 B per output element moved
    instead of 16.  tm_merge through the C ABI, median of `steps` calls."""
    from paper_1202_6575_gb300 import tm, workloads as W
    out = {"workload": "n = m = 2^28 int32 keys, no payloads", "unit": UNIT}
    for dist in ("uniform_1024", "uniform_full"):
        A, _, B, _ = W.large_merge(dist, False, dev)
        n, m = A.numel(), B.numel()
        C = torch.empty(n + m, dtype=torch.int32, device=dev)
        ws = tm.new_workspace(tm.tm_merge_workspace_size(n, m), dev)
        tm.tm_merge("i32", A, None, B, None, C, None, ws)
        ts = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            tm.tm_merge("i32", A, None, B, None, C, None, ws)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        assert tm.tm_read_status(ws) == 0
        ms = float(np.median(ts))
        gbs = (n + m) * 8 / (ms / 1e3) / 1e9
        out[dist] = {"ms": ms, "value": (n + m) / (ms / 1e3), "gbs": gbs, "frac_of_hbm": gbs / measured_peaks()[0]}
        del A, B, C, ws
        torch.cuda.empty_cache()
    return out


def bench_payload64(dev, steps: int = 10):
    """8-byte payload words (tm_config.payload_bytes = 8): n = m = 2**28 int32
    keys uniform over int32 with 64-bit payloads, tm_merge through the C ABI,
    median of `steps` calls; 24 B per output element (4 + 8 read, 4 + 8
    written)."""
    from paper_1202_6575_gb300 import tm, workloads as W
    A, Av, B, Bv = W.large_merge("uniform_full", False, dev)
    Aw, Bw = W.widen_payload(Av), W.widen_payload(Bv)
    del Av, Bv
    n, m = A.numel(), B.numel()
    C = torch.empty(n + m, dtype=torch.int32, device=dev)
    Cw = torch.empty(n + m, dtype=torch.int64, device=dev)
    ws = tm.new_workspace(tm.tm_merge_workspace_size(n, m), dev)
    tm.tm_merge("i32", A, Aw, B, Bw, C, Cw, ws)
    ts = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        tm.tm_merge("i32", A, Aw, B, Bw, C, Cw, ws)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    assert tm.tm_read_status(ws) == 0
    ms = float(np.median(ts))
    gbs = (n + m) * 24 / (ms / 1e3) / 1e9
    out = {"workload": "n = m = 2^28 int32 keys (uniform over int32) + 8-byte payloads", "unit": UNIT,
           "ms": ms, "value": (n + m) / (ms / 1e3), "gbs": gbs, "frac_of_hbm": gbs / measured_peaks()[0]}
    del A, Aw, B, Bw, C, Cw, ws
    torch.cuda.empty_cache()
    return out


def bench_batched(dev, steps: int = 10, pairs: int = 65536, with_plain: bool = True, cfg=None):
    """Batched form: 65,536 independent pairs (lengths log-uniform in
    [1, 2**16] per side, u64 keys + u32 payloads), autotuned, captured in a
    CUDA graph, replayed `steps` times.  Compared with the plain form: the
    same pairs as 65,536 tm_merge calls on one stream."""
    from paper_1202_6575_gb300 import tm, workloads as W
    a_off, A, Av, b_off, B, Bv = W.batched_pairs(dev, pairs=pairs)
    pairs = a_off.numel() - 1
    ta, tb = A.numel(), B.numel()
    total = ta + tb
    C = torch.empty(total, dtype=torch.int64, device=dev)
    Cv = torch.empty(total, dtype=torch.int32, device=dev)
    big = max(tm.tm_merge_batched_workspace_size(pairs, ta, tb, {"tile": t}) for t in (1024, 2048, 4096))
    ws = tm.new_workspace(big, dev)
    s = side_stream(dev)
    best = cfg or tm.tm_autotune_batched("u64", a_off, A, Av, b_off, B, Bv, C, Cv, ws, stream=s)
    tm.tm_merge_batched("u64", a_off, A, Av, b_off, B, Bv, C, Cv, ws, cfg=best, stream=s)
    s.synchronize()
    with tm.Graph(s) as g:
        tm.tm_merge_batched("u64", a_off, A, Av, b_off, B, Bv, C, Cv, ws, cfg=best, stream=s)
    for _ in range(2):
        g.launch()
    s.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        g.launch()
    e1.record(s)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    assert tm.tm_read_status(ws, stream=s) == 0
    ms_plain = None
    same = None
    if with_plain:
        # plain form: one tm_merge per pair (host loop, one stream)
        ho_a, ho_b = a_off.cpu().tolist(), b_off.cpu().tolist()
        wsp = tm.new_workspace(tm.tm_merge_workspace_size(1 << 16, 1 << 16), dev)
        def plain():
            for k in range(pairs):
                a0, a1, b0, b1 = ho_a[k], ho_a[k + 1], ho_b[k], ho_b[k + 1]
                c0 = a0 + b0
                L = (a1 - a0) + (b1 - b0)
                tm.tm_merge("u64", A[a0:a1], Av[a0:a1], B[b0:b1], Bv[b0:b1], C[c0:c0 + L], Cv[c0:c0 + L], wsp, stream=s)
        ref = (C.clone(), Cv.clone())                 # the graph's output
        C.fill_(-1)
        Cv.fill_(-1)
        s.wait_stream(torch.cuda.current_stream(dev))  # the merges on s write after the fills
        plain()
        s.synchronize()
        same = bool(torch.equal(ref[0], C) and torch.equal(ref[1], Cv))
        e0.record(s)
        plain()
        e1.record(s)
        e1.synchronize()
        ms_plain = e0.elapsed_time(e1)
    gbs = total * 24 / (ms / 1e3) / 1e9
    return {"workload": f"{pairs:,} pairs, lengths log-uniform in [1, 2^16] per side, u64 keys in [0, 2^20) + u32 "
                        f"payloads; {'fixed configuration' if cfg else 'autotuned'}; one CUDA graph (count, scan, "
                        "search, plan, persistent merge)",
            "elements": total, "value": total / (ms / 1e3), "unit": UNIT, "ms": ms, "steps": steps,
            "config": best, "gbs": gbs, "frac_of_hbm": gbs / measured_peaks()[0],
            "plain_per_pair_tm_merge": None if ms_plain is None else {"value": total / (ms_plain / 1e3),
                                                                       "ms": ms_plain, "calls": pairs},
            "speedup_vs_plain": None if ms_plain is None else ms_plain / ms,
            "bit_exact": same}


def bench_sort(dev, steps: int = 3, cfg=None, log2n: int = 28):
    """Stable merge sort of 2**28 u64 keys uniform in [0, 2**24) with u32
    payloads (original index): sorted runs of 4096, then 16 merge rounds.
    (log2n < 28: a smaller case of the same kernels, for profiles.)"""
    from paper_1202_6575_gb300 import tm, workloads as W
    src_k, src_v = W.sort_input(dev, n=1 << log2n)
    n = src_k.numel()
    keys, vals = torch.empty_like(src_k), torch.empty_like(src_v)
    tk, tv = torch.empty_like(src_k), torch.empty_like(src_v)
    big = max(tm.tm_merge_sort_workspace_size(n, {"tile": t}) for t in (1024, 2048, 4096))
    ws = tm.new_workspace(big, dev)
    s = side_stream(dev)
    best = cfg or tm.tm_autotune_sort("u64", src_k, src_v, keys, vals, tk, tv, ws, stream=s)
    times = []
    for _ in range(steps + 1):
        keys.copy_(src_k)
        vals.copy_(src_v)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        tm.tm_merge_sort("u64", keys, vals, tk, tv, ws, cfg=best, stream=s)
        e1.record(s)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    assert tm.tm_read_status(ws, stream=s) == 0
    ms = float(np.median(times[1:]))
    ref = (keys.clone(), vals.clone())
    # the same sort with two rounds per pass (cfg merge_ways = 4, tile 4096)
    ucfg = {"tile": 4096, "merge_ways": 4}
    utimes = []
    for _ in range(steps + 1):
        keys.copy_(src_k)
        vals.copy_(src_v)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        tm.tm_merge_sort("u64", keys, vals, tk, tv, ws, cfg=ucfg, stream=s)
        e1.record(s)
        e1.synchronize()
        utimes.append(e0.elapsed_time(e1))
    assert tm.tm_read_status(ws, stream=s) == 0
    same = bool(torch.equal(ref[0], keys) and torch.equal(ref[1], vals))
    # the stable order at full size: keys non-decreasing, and on equal keys
    # the payloads (original indices) increasing
    k0, k1, v0, v1 = ref[0][:-1], ref[0][1:], ref[1][:-1], ref[1][1:]
    stable = bool(((k0 < k1) | ((k0 == k1) & (v0 < v1))).all())
    idx = ref[1].long()                               # a permutation, each key its input's
    stable = stable and bool(torch.equal(torch.sort(idx).values, torch.arange(n, device=dev))) and \
        bool(torch.equal(ref[0], src_k[idx]))
    del k0, k1, v0, v1, idx
    ums = float(np.median(utimes[1:]))
    rounds = 0
    r = SORT_RUN
    while r < n:
        r *= 2
        rounds += 1
    moved = n * 24 * (rounds + 1)                     # run formation + every round read and write 12 B
    return {"workload": f"stable merge sort of 2^{log2n} u64 keys uniform in [0, 2^24) + u32 payloads",
            "elements": n, "value": n / (ms / 1e3), "unit": "sorted elems/s", "ms": ms, "rounds": rounds,
            "config": best, "passes_gbs": moved / (ms / 1e3) / 1e9,
            "frac_of_hbm": moved / (ms / 1e3) / 1e9 / measured_peaks()[0],
            "four_way_ms": ums, "four_way_passes": 1 + rounds // 2 + rounds % 2,
            "four_way_bit_exact": same, "bit_exact": bool(stable and same)}


def bench_segmented(dev, steps: int = 3):
    """Segmented stable sort: 65,536 segments whose lengths are those of the
    batched workload's pairs (n_k + m_k, each side log-uniform in [1, 2**16]),
    u64 keys uniform in [0, 2**20) (unsorted) with u32 payloads = index; one
    tm_merge_sort_segmented call, median of `steps` after one warm call.
    Checked at full size: inside every segment the keys are non-decreasing
    and equal keys keep their input order, and the output is a permutation
    that never moves an element out of its segment."""
    from paper_1202_6575_gb300 import tm, workloads as W
    a_off, A, Av, b_off, B, Bv = W.batched_pairs(dev)
    del A, Av, B, Bv
    a_off, b_off = a_off.cpu(), b_off.cpu()
    lens = (a_off[1:] - a_off[:-1]) + (b_off[1:] - b_off[:-1])
    offs = torch.cat([torch.zeros(1, dtype=torch.int64), torch.cumsum(lens, 0)])
    n = int(offs[-1])
    g = torch.Generator(device=dev)
    g.manual_seed(W.SEED_BASE + 9)
    src_k = torch.randint(0, 1 << 20, (n,), generator=g, device=dev, dtype=torch.int64)
    src_v = torch.arange(n, device=dev, dtype=torch.int64).to(torch.int32)
    keys, vals = torch.empty_like(src_k), torch.empty_like(src_v)
    tk, tv = torch.empty_like(src_k), torch.empty_like(src_v)
    ws = tm.new_workspace(tm.tm_merge_sort_segmented_workspace_size(n, offs), dev)
    times = []
    for _ in range(steps + 1):
        keys.copy_(src_k)
        vals.copy_(src_v)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        tm.tm_merge_sort_segmented("u64", keys, vals, offs, tk, tv, ws)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    assert tm.tm_read_status(ws) == 0
    ms = float(np.median(times[1:]))
    seg = torch.repeat_interleave(torch.arange(lens.numel(), device=dev), lens.to(dev))
    idx = vals.long()
    ok = bool(torch.equal(torch.sort(idx).values, torch.arange(n, device=dev))) and \
        bool(torch.equal(keys, src_k[idx])) and bool(torch.equal(seg[idx], seg))
    s0, s1, k0, k1, v0, v1 = seg[:-1], seg[1:], keys[:-1], keys[1:], vals[:-1], vals[1:]
    ok = ok and bool(((s0 != s1) | (k0 < k1) | ((k0 == k1) & (v0 < v1))).all())
    rounds = 0
    while (SORT_RUN << rounds) < int(lens.max()):
        rounds += 1
    moved = n * 24 * (rounds + 1)
    gbs = moved / (ms / 1e3) / 1e9
    return {"workload": f"{lens.numel():,} segments (lengths of the batched pairs), {n:,} u64 keys in [0, 2^20) + "
                        "u32 payloads, unsorted", "elements": n, "value": n / (ms / 1e3), "unit": "sorted elems/s",
            "ms": ms, "rounds": rounds, "passes_gbs": gbs, "frac_of_hbm": gbs / measured_peaks()[0],
            "bit_exact": ok}


def bench_learned(dev, merges: int = 256, log2_base: int = 28, log2_batch: int = 20):
    """LSM-style repeated merging: a sorted float32 base of 2**28 keys (3
    lognormals, mu 0/2/5, sigma 0.5) merged `merges` times with sorted
    batches of 2**20 keys from the same mixture (the base on the A side).
    Plain form: tm_cross_ranks + plan + tile merge per merge.  Learned form:
    the model (4096 segments + MLP 2-64-1) trained on 2**18 exact rank_high
    labels from the plain search, then tm_cross_ranks_learned (advancing the
    knot ranks) + plan + tile merge per merge.  Both end in bit-identical
    bases."""
    from paper_1202_6575_gb300 import tm, workloads as W
    N0, m = 1 << log2_base, 1 << log2_batch
    cap = N0 + merges * m
    X0, X0v = W.lsm_base(dev, n=N0)
    batches = [W.lsm_batch(k, dev, size=m, base_n=N0) for k in range(merges)]
    bufs = [(torch.empty(cap, dtype=torch.float32, device=dev), torch.empty(cap, dtype=torch.int32, device=dev))
            for _ in range(2)]
    p_max = tm.tm_merge_blocks(cap, m)
    xbar = torch.empty(p_max + 1, dtype=torch.int64, device=dev)
    ybar = torch.empty(p_max + 1, dtype=torch.int64, device=dev)
    tiles = torch.empty(2 * p_max * tm.tm_tile_record_bytes(), dtype=torch.uint8, device=dev)
    control = torch.zeros(256, dtype=torch.uint8, device=dev)
    s = side_stream(dev)

    def run(search):
        bufs[0][0][:N0].copy_(X0)
        bufs[0][1][:N0].copy_(X0v)
        torch.cuda.synchronize(dev)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(merges)]
        n = N0
        src = 0
        for k in range(merges):
            A, Av = bufs[src][0][:n], bufs[src][1][:n]
            B, Bv = batches[k]
            C, Cv = bufs[src ^ 1][0][:n + m], bufs[src ^ 1][1][:n + m]
            p = tm.tm_merge_blocks(n, m)
            ev[k][0].record(s)
            search(A, B, p)
            ev[k][1].record(s)
            tm.tm_plan_subproblems(n, m, p, xbar, ybar, tiles, stream=s)
            tm.tm_merge_tiles("f32", A, Av, B, Bv, tiles, tm.tm_plan_tile_count(n, m, p),
                              tm.tm_merge_tile_cap(n, m, p), C, Cv, control, stream=s)
            ev[k][2].record(s)
            n += m
            src ^= 1
        ev[-1][2].synchronize()
        assert tm.tm_read_status(control, stream=s) == 0
        total_ms = ev[0][0].elapsed_time(ev[-1][2])
        search_ms = [e[0].elapsed_time(e[1]) for e in ev]
        return total_ms, search_ms, src, n

    def plain(A, B, p):
        tm.tm_cross_ranks("f32", A, B, p, xbar, ybar, stream=s)

    run(plain)                                       # warm-up
    t_plain, srch_plain, src, n_final = run(plain)
    ref = bufs[src][0][:n_final].clone(), bufs[src][1][:n_final].clone()

    # model: trained on exact ranks of 2**18 mixture keys in the initial base
    t0 = time.perf_counter()
    q = W.lsm_label_keys(dev, count=1 << 18)
    labels = tm.tm_rank_search("f32", "high", q, X0)
    init = W.cdf_init(hidden=64)
    flat = torch.cat([init["W1"].reshape(-1), init["b1"], init["w2"], init["b2"].reshape(1)])
    model = tm.CdfModel(4096, 64, dev).init(X0, flat)
    model.train(q, labels, steps=400, lr=3e-3)
    qc = W.lsm_label_keys(dev, count=1 << 20, seed=W.SEED_BASE + 8)
    model.calibrate(qc, tm.tm_rank_search("f32", "high", qc, X0))
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    init_state = model.buf.clone()

    def learned(A, B, p):
        tm.tm_cross_ranks_learned(model, A, B, p, xbar, ybar, flags=tm.LEARNED_ADVANCE, stream=s)

    model.buf.copy_(init_state)
    run(learned)                                     # warm-up (advances the knot ranks)
    model.buf.copy_(init_state)
    torch.cuda.synchronize(dev)
    t_learned, srch_learned, src, n_final = run(learned)
    same = torch.equal(bufs[src][0][:n_final], ref[0]) and torch.equal(bufs[src][1][:n_final], ref[1])
    h = model.header()
    eps_s = model.eps_segments().cpu().numpy()
    # the same run with the model's piecewise-linear part alone (MLP output
    # 0: all network parameters zero), calibrated on the same keys
    pla = tm.CdfModel(4096, 64, dev).init(X0, torch.zeros_like(flat))
    pla.calibrate(qc, tm.tm_rank_search("f32", "high", qc, X0))
    pla_state = pla.buf.clone()

    def learned_pla(A, B, p):
        tm.tm_cross_ranks_learned(pla, A, B, p, xbar, ybar, flags=tm.LEARNED_ADVANCE, stream=s)

    run(learned_pla)                                 # warm-up
    pla.buf.copy_(pla_state)
    torch.cuda.synchronize(dev)
    t_pla, srch_pla, src, n_final = run(learned_pla)
    same_pla = torch.equal(bufs[src][0][:n_final], ref[0]) and torch.equal(bufs[src][1][:n_final], ref[1])
    hp = pla.header()
    eps_p = pla.eps_segments().cpu().numpy()
    elems = sum(N0 + k * m + m for k in range(merges))
    seg = (N0 + merges * m / 2) / 4096
    return {"workload": f"base 2^{log2_base} f32 (3 lognormals) merged {merges} times with sorted 2^{log2_batch} "
                        "batches; u32 payloads",
            "elements": elems,
            "plain": {"value": elems / (t_plain / 1e3), "unit": UNIT, "ms_total": t_plain,
                      "search_ms_mean": float(np.mean(srch_plain))},
            "learned": {"value": elems / (t_learned / 1e3), "unit": UNIT, "ms_total": t_learned,
                        "search_ms_mean": float(np.mean(srch_learned)),
                        "fallbacks": int(h["fallbacks"]), "learned_searches": int(h["learned"]),
                        "mean_window_probes": float(np.mean(np.log2(2 * (3 * eps_s * seg + 32) + 1))),
                        "plain_probes": float(np.log2(N0 + merges * m / 2)),
                        "train_seconds_once": train_s},
            "pla_only": {"value": elems / (t_pla / 1e3), "unit": UNIT, "ms_total": t_pla,
                         "search_ms_mean": float(np.mean(srch_pla)), "fallbacks": int(hp["fallbacks"]),
                         "mean_window_probes": float(np.mean(np.log2(2 * (3 * eps_p * seg + 32) + 1)))},
            "search_speedup": float(np.mean(srch_plain) / np.mean(srch_learned)),
            "search_speedup_pla_only": float(np.mean(srch_plain) / np.mean(srch_pla)),
            "mlp_vs_pla_search": float(np.mean(srch_pla) / np.mean(srch_learned)),
            "end_to_end_speedup": t_plain / t_learned,
            "end_to_end_speedup_pla_only": t_plain / t_pla,
            "bit_identical": bool(same and same_pla)}


def bench_search(dev, log2_base: int = 28, log2_batch: int = 20, reps: int = 30):
    """Steps 1-2 alone on the LSM inputs: one sorted float32 base (3
    lognormals) and one batch; the plain searches (tm_cross_ranks) vs the
    learned ones (tm_cross_ranks_learned, model trained as in the learned
    form), each launch after a 512 MB write that flushes L2; median of the
    launches after 3 warm-up ones (CUDA events)."""
    from paper_1202_6575_gb300 import tm, workloads as W
    n, m = 1 << log2_base, 1 << log2_batch
    A, _ = W.lsm_base(dev, n=n)
    B, _ = W.lsm_batch(0, dev, size=m, base_n=n)
    q = W.lsm_label_keys(dev, count=1 << 18)
    init = W.cdf_init(hidden=64)
    flat = torch.cat([init["W1"].reshape(-1), init["b1"], init["w2"], init["b2"].reshape(1)])
    model = tm.CdfModel(4096, 64, dev).init(A, flat)
    model.train(q, tm.tm_rank_search("f32", "high", q, A), steps=400, lr=3e-3)
    qc = W.lsm_label_keys(dev, count=1 << 20, seed=W.SEED_BASE + 8)
    model.calibrate(qc, tm.tm_rank_search("f32", "high", qc, A))
    p = tm.tm_merge_blocks(n, m)
    xbar = torch.empty(p + 1, dtype=torch.int64, device=dev)
    ybar = torch.empty_like(xbar)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream(dev)

    def timed(fn):
        ts = []
        for r in range(reps):
            with torch.cuda.stream(s):                 # on the timed stream: the flush ends before e0,
                flush.fill_(r & 255)                   # and the search is enqueued while it runs
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fn()
            e1.record(s)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
        return float(np.median(ts[3:]))

    plain_us = timed(lambda: tm.tm_cross_ranks("f32", A, B, p, xbar, ybar, stream=s))
    xp, yp = xbar.clone(), ybar.clone()
    learned_us = timed(lambda: tm.tm_cross_ranks_learned(model, A, B, p, xbar, ybar, stream=s))
    same = bool(torch.equal(xp, xbar) and torch.equal(yp, ybar))
    pla = tm.CdfModel(4096, 64, dev).init(A, torch.zeros_like(flat))      # the network's output 0
    pla.calibrate(qc, tm.tm_rank_search("f32", "high", qc, A))
    pla_us = timed(lambda: tm.tm_cross_ranks_learned(pla, A, B, p, xbar, ybar, stream=s))
    same = same and bool(torch.equal(xp, xbar) and torch.equal(yp, ybar))
    return {"workload": f"base 2^{log2_base} f32 (3 lognormals), batch 2^{log2_batch}, p = {p}",
            "plain_us": plain_us, "learned_us": learned_us, "pla_only_us": pla_us,
            "speedup": plain_us / learned_us, "speedup_pla_only": plain_us / pla_us,
            "mlp_vs_pla": pla_us / learned_us, "identical": same,
            "fallbacks": int(model.header()["fallbacks"]), "fallbacks_pla_only": int(pla.header()["fallbacks"])}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--stages", type=int, default=0)
    ap.add_argument("--split", type=int, default=0, help="in-CTA split: 1 blocks (paper's rule), 2 diagonal")
    ap.add_argument("--log2n", type=int, default=28, help="smaller cases for profiling only")
    ap.add_argument("--dists", default="", help="comma list of distributions (default: all four)")
    ap.add_argument("--no-skewed", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched, merge-sort and learned forms")
    ap.add_argument("--serial", action="store_true",
                    help="run each merge's search, plan and merge back to back on one stream (no overlap)")
    ap.add_argument("--form", default="", choices=["", "batched", "sort", "learned", "small", "search", "keys",
                                                   "partition", "payload64", "segmented"],
                    help="run one form alone (profiling)")
    ap.add_argument("--merges", type=int, default=256, help="learned form: merges (profiling)")
    ap.add_argument("--pairs", type=int, default=65536, help="batched form: pairs (profiling)")
    ap.add_argument("--log2-base", type=int, default=28, help="learned form: base size (profiling)")
    args = ap.parse_args()
    args.dists = [d for d in args.dists.split(",") if d] or None
    rank, local_rank, world = env_rank()

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    if args.form:
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        import __graft_entry__
        __graft_entry__.build()
        if args.form == "batched":
            fixed = {k: v for k, v in (("tile", args.tile), ("threads", args.threads), ("stages", args.stages),
                                       ("split", args.split)) if v} or None
            out = bench_batched(dev, pairs=args.pairs, with_plain=args.pairs == 65536 and fixed is None, cfg=fixed)
        elif args.form == "sort":
            fixed = {k: v for k, v in (("tile", args.tile), ("threads", args.threads), ("stages", args.stages),
                                       ("split", args.split)) if v} or None
            out = bench_sort(dev, cfg=fixed, log2n=args.log2n)
        elif args.form == "small":
            out = bench_small_merge(dev)
        elif args.form == "search":
            out = bench_search(dev, log2_base=args.log2_base)
        elif args.form == "keys":
            out = bench_keys_only(dev)
        elif args.form == "partition":
            out = bench_partition(dev)
        elif args.form == "payload64":
            out = bench_payload64(dev)
        elif args.form == "segmented":
            out = bench_segmented(dev)
        else:
            out = bench_learned(dev, merges=args.merges, log2_base=args.log2_base)
        print(json.dumps({"form": args.form, **out}), flush=True)
        return

    import torch.distributed as dist
    if world > 1:
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)

    import __graft_entry__
    __graft_entry__.build()
    from paper_1202_6575_gb300 import tm

    cfg = {}
    if args.tile:
        cfg["tile"] = args.tile
    if args.threads:
        cfg["threads"] = args.threads
    if args.stages:
        cfg["stages"] = args.stages
    if args.split:
        cfg["split"] = args.split
    cfg = cfg or None

    items = make_inputs(dev, args.log2n, args.dists, not args.no_skewed)
    for it in items:
        n, m = it["A"].numel(), it["B"].numel()
        it["n"], it["m"] = n, m
        it["p"] = tm.tm_merge_blocks(n, m, cfg)
        it["xbar"] = torch.empty(it["p"] + 1, dtype=torch.int64, device=dev)
        it["ybar"] = torch.empty(it["p"] + 1, dtype=torch.int64, device=dev)
        it["tiles"] = torch.empty(2 * it["p"] * tm.tm_tile_record_bytes(), dtype=torch.uint8, device=dev)
        it["cap"] = tm.tm_merge_tile_cap(n, m, it["p"])
        it["count"] = tm.tm_plan_tile_count(n, m, it["p"])
    control = torch.zeros(256, dtype=torch.uint8, device=dev)
    cmax = max(it["n"] + it["m"] for it in items)
    C = torch.empty(cmax, dtype=torch.int32, device=dev)
    Cv = torch.empty(cmax, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    elems_per_step = sum(it["n"] + it["m"] for it in items)
    bytes_merge_per_step = sum(2 * (it["n"] + it["m"]) * 8 for it in items)
    # algorithmic search bytes: ceil(log2(len + 1)) probes of 4 B per search,
    # p searches into each array
    search_bytes_per_step = sum(it["p"] * 4 * (int(it["n"]).bit_length() + int(it["m"]).bit_length())
                                for it in items)

    # Steps 1-2 and the selection of every merge run on a second stream, ahead
    # of the merges on `stream`: merge k waits for its own records only, so
    # the searches and plans of the later merges overlap the earlier merges
    # (the eight merges are independent).  A merge's records are rewritten
    # by the next step only after that merge has read them.  --serial runs
    # every merge's three phases back to back on one stream instead.
    s_side = side_stream(dev)
    merged_ev = [None] * len(items)

    # per-merge events: search start, plan start, plan end (on s_plan), merge
    # start, merge end (on stream)
    def step(evs=None, serial=args.serial):
        s_plan = stream if serial else s_side
        ready = []
        for k, it in enumerate(items):
            n, m, p = it["n"], it["m"], it["p"]
            if merged_ev[k] is not None and s_plan is not stream:
                s_plan.wait_event(merged_ev[k])
            if evs is not None:
                evs[k][0].record(s_plan)
            tm.tm_cross_ranks("i32", it["A"], it["B"], p, it["xbar"], it["ybar"], stream=s_plan)
            if evs is not None:
                evs[k][1].record(s_plan)
            tm.tm_plan_subproblems(n, m, p, it["xbar"], it["ybar"], it["tiles"], cfg=cfg, stream=s_plan)
            if evs is not None:
                evs[k][2].record(s_plan)
            if s_plan is stream:
                merge_one(k, it, evs)
            else:
                r = torch.cuda.Event()
                r.record(s_plan)
                ready.append(r)
        for k, it in enumerate(items if s_plan is not stream else []):
            stream.wait_event(ready[k])
            merge_one(k, it, evs)

    def merge_one(k, it, evs):
        n, m = it["n"], it["m"]
        if evs is not None:
            evs[k][3].record(stream)
        tm.tm_merge_tiles("i32", it["A"], it["Av"], it["B"], it["Bv"], it["tiles"], it["count"], it["cap"],
                          C[:n + m], Cv[:n + m], control, cfg=cfg, stream=stream)
        if evs is not None:
            evs[k][4].record(stream)
        d = torch.cuda.Event()
        d.record(stream)
        merged_ev[k] = d

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    assert tm.tm_read_status(control) == 0

    evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in items] for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with sampler:
        t_start.record(stream)
        s_side.wait_event(t_start)
        for s in range(args.steps):
            step(evs[s])
        t_end.record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    elapsed_ms = t_start.elapsed_time(t_end)
    assert tm.tm_read_status(control) == 0
    # the merge kernel alone: a few steps with the phases back to back
    evs_alone = [[[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in items] for _ in range(3)]
    for s in range(3):
        step(evs_alone[s], serial=True)
    torch.cuda.synchronize(dev)
    assert tm.tm_read_status(control) == 0
    merge_alone_ms = sum(e[3].elapsed_time(e[4]) for st in evs_alone for e in st) / 3
    search_ms = sum(e[0].elapsed_time(e[1]) for st in evs for e in st)
    plan_ms = sum(e[1].elapsed_time(e[2]) for st in evs for e in st)
    merge_ms = sum(e[3].elapsed_time(e[4]) for st in evs for e in st)
    per_item_merge_ms = {it["name"]: float(np.mean([evs[s][k][3].elapsed_time(evs[s][k][4]) for s in range(args.steps)]))
                         for k, it in enumerate(items)}

    elapsed_max = max_over_ranks(elapsed_ms, dev)
    value = whole_job_rate(elems_per_step * args.steps, world, elapsed_max)

    peak, peak_kind = measured_peaks()
    launches = len(items) * args.steps
    achieved = (bytes_merge_per_step * args.steps / launches) / ((merge_ms / launches) / 1e3) / 1e9
    traffic_per_elem, traffic_src = profile_traffic("merge_engine_kernel")
    traffic = None if traffic_per_elem is None else traffic_per_elem * elems_per_step / len(items)
    roofline = {"bound": "hbm", "kernel": "merge_engine_kernel", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs (copy)",
                "traffic": traffic, "traffic_source": traffic_src,
                "algorithmic_bytes_per_launch": bytes_merge_per_step / len(items),
                # kernel time of the searches and plans against all three
                # (with the overlap they run beside the merges)
                "search_share": search_ms / (search_ms + plan_ms + merge_ms),
                "plan_share": plan_ms / (search_ms + plan_ms + merge_ms),
                "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                # the same kernel with no search or plan running beside it
                "frac_alone": bytes_merge_per_step / (merge_alone_ms / 1e3) / 1e9 / peak,
                # whole step: merge bytes plus the searches' probe bytes (one
                # 4-byte key per probe) over the step's wall time
                "step_frac": (bytes_merge_per_step + search_bytes_per_step) * args.steps /
                             (elapsed_ms / 1e3) / 1e9 / peak}

    # End to end: pinned host inputs -> device, merge through tm_merge, result
    # -> host, for every merge of the step.  Copies in, merges and copies out
    # run on three streams, pipelined across the eight merges and across
    # steps (merge k's output goes to one of two device buffers, reused by
    # merge k + 2 once its copy-out has finished; a step's copy into merge
    # k's inputs waits for the previous step's merge k).
    e2e = None
    cpu = None
    if not args.no_e2e:
        pin = lambda t: torch.empty(t.shape, dtype=t.dtype, pin_memory=True).copy_(t)
        for it in items:
            it["hA"], it["hAv"], it["hB"], it["hBv"] = (pin(it["A"]).numpy(), pin(it["Av"]).numpy(),
                                                        pin(it["B"]).numpy(), pin(it["Bv"]).numpy())
            it["hC"] = torch.empty(it["n"] + it["m"], dtype=torch.int32, pin_memory=True)
            it["hCv"] = torch.empty(it["n"] + it["m"], dtype=torch.int32, pin_memory=True)
        Cs = [(C, Cv), (torch.empty(cmax, dtype=torch.int32, device=dev), torch.empty(cmax, dtype=torch.int32, device=dev))]
        wss = [tm.new_workspace(max(tm.tm_merge_workspace_size(it["n"], it["m"], cfg) for it in items), dev)
               for _ in range(2)]
        s_in, s_comp, s_out = side_stream(dev), side_stream(dev), side_stream(dev)
        h2d = d2h = 0
        out_done = [None, None]
        merged = {}                       # per merge: its last tm_merge, which read the device inputs

        def e2e_step():
            nonlocal h2d, d2h
            h2d = d2h = 0
            for k, it in enumerate(items):
                n, m = it["n"], it["m"]
                if k in merged:               # the previous step's merge k has read these inputs
                    s_in.wait_event(merged[k])
                with torch.cuda.stream(s_in):
                    it["A"].copy_(torch.from_numpy(it["hA"]), non_blocking=True)
                    it["Av"].copy_(torch.from_numpy(it["hAv"]), non_blocking=True)
                    it["B"].copy_(torch.from_numpy(it["hB"]), non_blocking=True)
                    it["Bv"].copy_(torch.from_numpy(it["hBv"]), non_blocking=True)
                    ev_in = torch.cuda.Event()
                    ev_in.record(s_in)
                b = k % 2
                s_comp.wait_event(ev_in)
                if out_done[b] is not None:
                    s_comp.wait_event(out_done[b])
                Cb, Cvb = Cs[b]
                tm.tm_merge("i32", it["A"], it["Av"], it["B"], it["Bv"], Cb[:n + m], Cvb[:n + m], wss[b], cfg=cfg,
                            stream=s_comp)
                ev_c = torch.cuda.Event()
                ev_c.record(s_comp)
                merged[k] = ev_c
                s_out.wait_event(ev_c)
                with torch.cuda.stream(s_out):
                    it["hC"].copy_(Cb[:n + m], non_blocking=True)
                    it["hCv"].copy_(Cvb[:n + m], non_blocking=True)
                    out_done[b] = torch.cuda.Event()
                    out_done[b].record(s_out)
                h2d += 2 * (n + m) * 4
                d2h += 2 * (n + m) * 4

        e2e_step()
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s_in)
        for _ in range(args.e2e_steps):
            e2e_step()                         # copies in of the next step overlap this step's copies out
        s_in.wait_stream(s_out)
        e1.record(s_in)
        torch.cuda.synchronize(dev)
        te = max_over_ranks(e0.elapsed_time(e1), dev)
        e2e = {"value": whole_job_rate(elems_per_step * args.e2e_steps, world, te), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
               "path": "pinned host -> H2D (stream 1) -> tm_merge (C ABI, stream 2) -> D2H (stream 3) -> pinned "
                       "host, pipelined over the eight merges of a step and across steps"}
        for w in wss:
            assert tm.tm_read_status(w, stream=s_comp) == 0
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(items)

    clocks = sampler.summary(power_floor_w=200.0)
    forms = None
    n_merges, lengths, p_first = len(items), [(it["n"], it["m"]) for it in items], items[0]["p"]
    if not args.no_forms:
        for it in items:
            it.clear()
        torch.cuda.empty_cache()
        forms = {"merge_1m_p1024": bench_small_merge(dev), "batched": bench_batched(dev),
                 "merge_sort": bench_sort(dev), "keys_only": bench_keys_only(dev),
                 "payload64": bench_payload64(dev), "segmented_sort": guarded(bench_segmented, dev),
                 "partition_ablation": bench_partition(dev)}
        torch.cuda.empty_cache()
        forms["learned"] = bench_learned(dev)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            forms["batched"]["cpu_baseline"] = guarded(cpu_batched_baseline)
            forms["merge_sort"]["cpu_baseline"] = guarded(cpu_sort_baseline)
            forms["learned"]["cpu_baseline"] = guarded(cpu_learned_baseline)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": elapsed_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
                "data": "synthetic",
                "config": headline_config(args, world, lengths, p_first),
                "forms": forms,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": 3 * n_merges * args.steps}
        # Every figure first, on a line of its own that is not JSON; then the
        # result line, short enough to survive a truncated log.
        detail = dict(line, per_merge_ms=per_item_merge_ms, config=dict(line["config"], workload=WORKLOAD))
        print("detail " + json.dumps(detail), flush=True)
        print(json.dumps(compact_line(line, peak), separators=(",", ":")), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
