"""Seeded random sweep of the merge, the merge sort and the segmented sort
against the oracle: key types, payload widths (none, 4 and 8 bytes),
launch configurations, tie-heavy and tie-free keys, and sizes drawn both
at random and next to the run, tile and block boundaries.  Every output
element is compared; each case prints its seed in the failure message."""
import numpy as np
import pytest
import torch

import oracle
from paper_1202_6575_gb300 import tm, workloads as W
from tests.helpers import first_mismatch, to_np, vals_np

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

KTS = ["u32", "i32", "u64", "f32"]
MERGE_CFGS = [None, {"tile": 1024}, {"tile": 4096, "threads": 256}, {"split": 1}, "few_blocks",
              {"partition": 1}, {"unfused": 1}]
SORT_CFGS = [None, {"tile": 1024}, {"tile": 4096, "threads": 256, "stages": 3}, {"merge_ways": 4},
             {"split": 1, "tile": 2048}]
EDGES = [0, 1, 2, 31, 1023, 1024, 1025, 2047, 2048, 2049, 4095, 4096, 4097, 8191, 8192, 8193, 16385, 65536]


def draw_size(rng, hi):
    if rng.random() < 0.4:
        return int(min(hi, EDGES[rng.integers(len(EDGES))] * (1 + int(rng.integers(0, 3)))))
    return int(rng.integers(0, hi + 1))


def keys_of(rng, n, kt):
    """Unsorted keys of type kt as a CPU tensor: few distinct values or
    many, sometimes including the type's extreme values."""
    alphabet = [1, 3, 50, 1 << 12, None][rng.integers(5)]
    if kt == "f32":
        if alphabet is None:
            k = rng.standard_normal(n).astype(np.float32) * 1e3
        else:
            k = (rng.integers(-alphabet, alphabet + 1, n) * 0.5).astype(np.float32)
            k[rng.random(n) < 0.05] = -0.0                 # equal to +0.0
        return torch.from_numpy(k)
    if kt == "u64":
        k = rng.integers(0, 1 << 63, n, dtype=np.uint64) if alphabet is None else \
            rng.integers(0, alphabet, n, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15 & ((1 << 58) - 1))
        if alphabet is None and n:
            k[rng.integers(0, n, max(1, n // 100))] = np.uint64((1 << 64) - 1)
        return torch.from_numpy(k.view(np.int64))
    if kt == "u32":
        k = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32) if alphabet is None else \
            (rng.integers(0, alphabet, n, dtype=np.uint64) * 77777).astype(np.uint32)
        if alphabet is None and n:
            k[rng.integers(0, n, max(1, n // 100))] = np.uint32(0xFFFFFFFF)
        return torch.from_numpy(k.view(np.int32))
    k = rng.integers(-(1 << 31), 1 << 31, n, dtype=np.int64).astype(np.int32) if alphabet is None else \
        (rng.integers(-alphabet, alphabet, n) * 1001).astype(np.int32)
    return torch.from_numpy(k)


def sorted_keys(k, kt):
    return torch.from_numpy(np.sort(to_np(k, kt), kind="stable").view(k.numpy().dtype))


def payload_for(n, width, src):
    tags = W.payload(src, n, "cpu")
    return tags, (None if width == 0 else (tags if width == 4 else W.widen_payload(tags)))


def check_payloads(got, want_tags, width, where):
    if width == 0:
        assert got is None, where
        return
    g = got.cpu().numpy().view(np.uint32 if width == 4 else np.uint64)
    w = want_tags if width == 4 else \
        W.widen_payload(torch.from_numpy(want_tags.view(np.int32))).numpy().view(np.uint64)
    assert first_mismatch(g, w) is None, f"{where}: payload mismatch at {first_mismatch(g, w)}"


@pytest.mark.parametrize("case", range(40))
def test_merge_sweep(case):
    rng = np.random.default_rng(7000 + case)
    kt = KTS[case % 4]
    n, m = draw_size(rng, 300000), draw_size(rng, 300000)
    width = [0, 4, 8][rng.integers(3)]
    cfg = MERGE_CFGS[rng.integers(len(MERGE_CFGS))]
    if cfg == "few_blocks":                             # fewer, larger blocks than the default (within a tile)
        cfg = {"p": max(1, (n + m) // 1500 + int(rng.integers(0, 3)))}
    if width != 4 and cfg is not None and "split" in cfg:
        cfg = None                                      # the sweep takes the paper's in-CTA rule with 4-byte payloads
    A, B = sorted_keys(keys_of(rng, n, kt), kt), sorted_keys(keys_of(rng, m, kt), kt)
    ta, Av = payload_for(n, width, 0)
    tb, Bv = payload_for(m, width, 1)
    where = f"case {case}: {kt} n={n} m={m} payload={width} cfg={cfg}"
    d = lambda t: None if t is None else t.to(DEV)
    C, Cv, ws = tm.tm_merge(kt, d(A), d(Av), d(B), d(Bv), cfg=cfg)
    assert tm.tm_read_status(ws) == 0, where
    K, V = oracle.merge_two_pointer(to_np(A, kt), vals_np(ta), to_np(B, kt), vals_np(tb))
    assert first_mismatch(to_np(C, kt), K) is None, f"{where}: key mismatch at {first_mismatch(to_np(C, kt), K)}"
    check_payloads(Cv, V, width, where)


@pytest.mark.parametrize("case", range(40))
def test_sort_sweep(case):
    rng = np.random.default_rng(9000 + case)
    kt = KTS[case % 4]
    n = draw_size(rng, 400000)
    width = [0, 4, 8][rng.integers(3)]
    cfg = SORT_CFGS[rng.integers(len(SORT_CFGS))]
    if width != 4 and cfg is not None and cfg.get("split") == 1:
        cfg = None
    keys = keys_of(rng, n, kt)
    tags, vals = payload_for(n, width, 0)
    where = f"case {case}: {kt} n={n} payload={width} cfg={cfg}"
    K, V, ws = tm.tm_merge_sort(kt, keys.to(DEV).clone(), None if vals is None else vals.to(DEV).clone(), cfg=cfg)
    assert tm.tm_read_status(ws) == 0, where
    OK, OV = oracle.merge_sort(to_np(keys, kt), vals_np(tags), run=32)
    assert first_mismatch(to_np(K, kt), OK) is None, f"{where}: key mismatch at {first_mismatch(to_np(K, kt), OK)}"
    check_payloads(V, OV, width, where)


@pytest.mark.parametrize("case", range(16))
def test_segmented_sort_sweep(case):
    rng = np.random.default_rng(11000 + case)
    kt = KTS[case % 4]
    segs = int(rng.integers(1, 60))
    lens = [draw_size(rng, 20000) for _ in range(segs)]
    n = sum(lens)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    width = [0, 4, 8][rng.integers(3)]
    keys = keys_of(rng, n, kt)
    tags, vals = payload_for(n, width, 0)
    where = f"case {case}: {kt} segments={segs} n={n} payload={width}"
    K, V, ws = tm.tm_merge_sort_segmented(kt, keys.to(DEV).clone(), None if vals is None else vals.to(DEV).clone(),
                                          off)
    assert tm.tm_read_status(ws) == 0, where
    hk, ht = to_np(keys, kt), vals_np(tags)
    OK = np.empty_like(hk)
    OV = np.empty_like(ht)
    for q in range(segs):
        a, b = off[q], off[q + 1]
        OK[a:b], OV[a:b] = oracle.merge_sort(hk[a:b], ht[a:b], run=32)
    assert first_mismatch(to_np(K, kt), OK) is None, f"{where}: key mismatch at {first_mismatch(to_np(K, kt), OK)}"
    check_payloads(V, OV, width, where)
