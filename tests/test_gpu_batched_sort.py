"""GPU parity of the batched merge and the stable merge sort (Section 3)
against the CPU oracle, bit-exact (keys and tagged payloads)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1202_6575_gb300 import tm, workloads as W
from tests.helpers import first_mismatch, to_np, vals_np

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def batched_check(a_off, A, Av, b_off, B, Bv, kt="u64", cfg=None, C=None, Cv=None, run=None):
    dev = lambda t: t.to(DEV)
    if run is None:
        C, Cv, ws = tm.tm_merge_batched(kt, dev(a_off), dev(A), dev(Av), dev(b_off), dev(B), dev(Bv), cfg=cfg)
        assert tm.tm_read_status(ws) == 0
    K, V = oracle.merge_batched(a_off.cpu().numpy(), to_np(A, kt), vals_np(Av), b_off.cpu().numpy(),
                                to_np(B, kt), vals_np(Bv))
    ck, cv = to_np(C, kt), vals_np(Cv)
    assert first_mismatch(ck, K) is None, f"key mismatch at {first_mismatch(ck, K)}"
    assert first_mismatch(cv, V) is None, f"payload mismatch at {first_mismatch(cv, V)}"


def csr_pairs(lens_a, lens_b, kt, seed, alphabet=1 << 20):
    rng = np.random.default_rng(seed)
    a_off = np.concatenate([[0], np.cumsum(lens_a)]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(lens_b)]).astype(np.int64)
    dt = {"u64": np.uint64, "u32": np.uint32, "i32": np.int32, "f32": np.float32}[kt]
    parts_a = [np.sort(rng.integers(0, alphabet, int(k))).astype(dt) for k in lens_a]
    parts_b = [np.sort(rng.integers(0, alphabet, int(k))).astype(dt) for k in lens_b]
    A = np.concatenate(parts_a) if len(parts_a) else np.empty(0, dt)
    B = np.concatenate(parts_b) if len(parts_b) else np.empty(0, dt)
    tA = torch.from_numpy(A.view(np.int64) if kt == "u64" else (A.view(np.int32) if kt in ("u32", "i32") else A))
    tB = torch.from_numpy(B.view(np.int64) if kt == "u64" else (B.view(np.int32) if kt in ("u32", "i32") else B))
    return (torch.from_numpy(a_off), tA, W.payload(0, len(A), "cpu"), torch.from_numpy(b_off), tB,
            W.payload(1, len(B), "cpu"))


@pytest.mark.parametrize("kt", ["u64", "u32", "i32", "f32"])
def test_batched_edge_pairs(kt):
    lens_a = [0, 0, 5, 1, 3000, 0, 7, 2048, 4096, 1, 10000]
    lens_b = [0, 4, 0, 1, 2, 3000, 7, 2048, 1, 9999, 3]
    batched_check(*csr_pairs(lens_a, lens_b, kt, 1, alphabet=50), kt=kt)
    batched_check(*csr_pairs(lens_a, lens_b, kt, 2), kt=kt, cfg={"tile": 512})


@pytest.mark.parametrize("split", [1, 2])
def test_batched_log_uniform_small(split):
    a_off, A, Av, b_off, B, Bv = W.batched_pairs("cpu", pairs=3000, log2_max=12)
    batched_check(a_off, A, Av, b_off, B, Bv, cfg={"split": split})


def test_batched_mostly_empty_pairs():
    """Long runs of empty pairs: a search/plan CTA can span more pairs than
    its shared-memory window holds and then finds its pairs in global memory."""
    rng = np.random.default_rng(4)
    pairs = 6000
    lens_a = np.where(rng.random(pairs) < 0.98, 0, rng.integers(1, 5000, pairs))
    lens_b = np.where(rng.random(pairs) < 0.98, 0, rng.integers(1, 5000, pairs))
    lens_a[:700] = 0
    lens_b[:700] = 0
    lens_a[1000] = 300000
    lens_a[2000:3000] = 0                   # 1000 empty pairs between two tiny ones: one CTA spans them
    lens_b[2000:3000] = 0
    lens_a[1999], lens_b[1999], lens_a[3000], lens_b[3000] = 3, 2, 4, 1
    batched_check(*csr_pairs(lens_a, lens_b, "u64", 9), kt="u64", cfg={"tile": 256})


def test_keys_only_batched_and_sort():
    a_off, A, Av, b_off, B, Bv = W.batched_pairs("cpu", pairs=2000, log2_max=12, seed=31)
    d = lambda t: t.to(DEV)
    C, Cv, ws = tm.tm_merge_batched("u64", d(a_off), d(A), None, d(b_off), d(B), None)
    assert Cv is None and tm.tm_read_status(ws) == 0
    K, _ = oracle.merge_batched(a_off.numpy(), to_np(A, "u64"), vals_np(Av), b_off.numpy(), to_np(B, "u64"),
                                vals_np(Bv))
    assert first_mismatch(to_np(C, "u64"), K) is None
    keys, vals = W.sort_input("cpu", n=(1 << 18) + 333, key_bits=12)
    sk, sv, ws = tm.tm_merge_sort("u64", keys.to(DEV).clone(), None)
    assert sv is None and tm.tm_read_status(ws) == 0
    assert np.array_equal(to_np(sk, "u64"), np.sort(to_np(keys, "u64"), kind="stable"))


def test_batched_no_pairs_and_all_empty():
    z = torch.zeros(1, dtype=torch.int64)
    e = torch.empty(0, dtype=torch.int64)
    ev = torch.empty(0, dtype=torch.int32)
    C, Cv, ws = tm.tm_merge_batched("u64", z.to(DEV), e.to(DEV), ev.to(DEV), z.to(DEV), e.to(DEV), ev.to(DEV))
    assert tm.tm_read_status(ws) == 0 and C.numel() == 0
    zz = torch.zeros(5, dtype=torch.int64)
    C, Cv, ws = tm.tm_merge_batched("u64", zz.to(DEV), e.to(DEV), ev.to(DEV), zz.to(DEV), e.to(DEV), ev.to(DEV))
    assert tm.tm_read_status(ws) == 0


def test_batched_in_cuda_graph_replayed():
    a_off, A, Av, b_off, B, Bv = W.batched_pairs("cpu", pairs=1000, log2_max=12, seed=77)
    d = [t.to(DEV) for t in (a_off, A, Av, b_off, B, Bv)]
    C = torch.empty(A.numel() + B.numel(), dtype=torch.int64, device=DEV)
    Cv = torch.empty(A.numel() + B.numel(), dtype=torch.int32, device=DEV)
    ws = tm.new_workspace(tm.tm_merge_batched_workspace_size(1000, A.numel(), B.numel()), DEV)
    s = torch.cuda.Stream()
    tm.tm_merge_batched("u64", *d, C=C, Cv=Cv, workspace=ws, stream=s)   # first call outside capture
    s.synchronize()
    with tm.Graph(s) as g:
        tm.tm_merge_batched("u64", *d, C=C, Cv=Cv, workspace=ws, stream=s)
    for _ in range(2):
        C.fill_(-1)
        Cv.fill_(-1)
        torch.cuda.synchronize()
        g.launch()
        s.synchronize()
        assert tm.tm_read_status(ws, stream=s) == 0
        batched_check(a_off, A, Av, b_off, B, Bv, C=C, Cv=Cv, run=False)


def test_autotune_batched_then_default_call():
    a_off, A, Av, b_off, B, Bv = W.batched_pairs("cpu", pairs=4000, log2_max=13, seed=5)
    d = [t.to(DEV) for t in (a_off, A, Av, b_off, B, Bv)]
    C = torch.empty(A.numel() + B.numel(), dtype=torch.int64, device=DEV)
    Cv = torch.empty_like(C, dtype=torch.int32)
    big = max(tm.tm_merge_batched_workspace_size(4000, A.numel(), B.numel(), {"tile": t}) for t in (1024, 2048, 4096))
    ws = tm.new_workspace(big, DEV)
    best = tm.tm_autotune_batched("u64", *d, C, Cv, ws)
    assert best["tile"] in (1024, 2048, 4096) and best["threads"] in (128, 256)
    C2, Cv2, ws2 = tm.tm_merge_batched("u64", *d, workspace=ws)          # cfg None: tuned choice
    assert tm.tm_read_status(ws2) == 0
    batched_check(a_off, A, Av, b_off, B, Bv, C=C2, Cv=Cv2, run=False)
    assert tm.tm_autotune_clear() >= 1


def test_batched_full_size():
    """65,536 pairs, lengths log-uniform in [1, 2**16] per side, u64 keys in
    [0, 2**20): the batched workload, every output element compared."""
    a_off, A, Av, b_off, B, Bv = W.batched_pairs(DEV)
    C, Cv, ws = tm.tm_merge_batched("u64", a_off, A, Av, b_off, B, Bv)
    assert tm.tm_read_status(ws) == 0
    K, V = oracle.merge_batched(a_off.cpu().numpy(), to_np(A, "u64"), vals_np(Av), b_off.cpu().numpy(),
                                to_np(B, "u64"), vals_np(Bv))
    ck, cv = to_np(C, "u64"), vals_np(Cv)
    assert first_mismatch(ck, K) is None and first_mismatch(cv, V) is None


# ---------------------------------------------------------------------------
# Merge sort
# ---------------------------------------------------------------------------

def sort_check(keys, vals, kt, cfg=None):
    dk, dv = keys.to(DEV).clone(), vals.to(DEV).clone()
    K, V, ws = tm.tm_merge_sort(kt, dk, dv, cfg=cfg)
    assert tm.tm_read_status(ws) == 0
    hk, hv = to_np(keys, kt), vals_np(vals)
    OK, OV = oracle.merge_sort(hk, hv, run=32)
    assert first_mismatch(to_np(K, kt), OK) is None, "keys"
    assert first_mismatch(vals_np(V), OV) is None, "payloads"


@pytest.mark.parametrize("n", [0, 1, 2, 1000, 1024, 1025, 4095, 4096, 4097, 8193, 65537, (1 << 20) + 3])
@pytest.mark.parametrize("kt", ["u64", "u32"])
def test_merge_sort_sizes(n, kt):
    g = torch.Generator().manual_seed(n)
    keys = torch.randint(0, 1 << 12, (n,), generator=g, dtype=torch.int64)
    keys = keys if kt == "u64" else keys.to(torch.int32)
    vals = torch.arange(n, dtype=torch.int64).to(torch.int32)
    sort_check(keys, vals, kt)


@pytest.mark.parametrize("kt", ["i32", "f32"])
def test_merge_sort_signed_and_float(kt):
    g = torch.Generator().manual_seed(3)
    n = 300001
    if kt == "i32":
        keys = torch.randint(-1000, 1000, (n,), generator=g, dtype=torch.int32)
    else:
        keys = (torch.randint(-50, 50, (n,), generator=g) * 0.5).to(torch.float32)
        keys[::7] = -0.0                         # -0.0 and +0.0 are equal keys
    vals = torch.arange(n, dtype=torch.int32)
    sort_check(keys, vals, kt)


@pytest.mark.parametrize("split", [1, 2])
def test_merge_sort_configs(split):
    keys, vals = W.sort_input("cpu", n=(1 << 18) + 77, key_bits=10)
    for tile in (1024, 4096):
        sort_check(keys, vals, "u64", cfg={"tile": tile, "split": split})


@pytest.mark.parametrize("n", [2049, 3 * 4096 + 5, 16384, 16385, 4 * 16384 - 1, 4 * 16384 + 1, 5 * 16384 + 3,
                               16 * 16384 + 1000])
@pytest.mark.parametrize("alphabet", [1, 3, 1 << 12])
def test_fused_sort_rounds_against_the_oracle(n, alphabet):
    """Two rounds fused into one pass (cfg merge_ways = 4: groups of four
    runs, some of them partial or empty at the end), with all keys equal,
    three distinct keys and many: the oracle's stable sort, as with one
    round per pass."""
    g = torch.Generator().manual_seed(n + alphabet)
    keys = torch.randint(0, alphabet, (n,), generator=g, dtype=torch.int64)
    vals = torch.arange(n, dtype=torch.int32)
    sort_check(keys, vals, "u64", cfg={"merge_ways": 4})
    sort_check(keys, vals, "u64")


@pytest.mark.parametrize("tile", [1024, 2048, 4096])
@pytest.mark.parametrize("kt", ["u32", "i32", "u64", "f32"])
def test_fused_sort_rounds_tiles_and_key_types(tile, kt):
    g = torch.Generator().manual_seed(tile)
    n = (1 << 17) + 12345
    keys = torch.randint(-300, 300, (n,), generator=g, dtype=torch.int64)
    keys = {"u64": keys + 300, "u32": (keys + 300).to(torch.int32), "i32": keys.to(torch.int32),
            "f32": (keys * 0.25).to(torch.float32)}[kt]
    vals = torch.arange(n, dtype=torch.int32)
    sort_check(keys, vals, kt, cfg={"tile": tile, "merge_ways": 4})


def test_fused_sort_rounds_keys_only():
    g = torch.Generator().manual_seed(9)
    n = (1 << 16) + 999
    keys = torch.randint(0, 1 << 10, (n,), generator=g, dtype=torch.int64)
    K, V, ws = tm.tm_merge_sort("u64", keys.to(DEV).clone(), None, cfg={"merge_ways": 4})
    assert V is None and tm.tm_read_status(ws) == 0
    OK, _ = oracle.merge_sort(to_np(keys, "u64"), np.arange(n, dtype=np.uint32), run=32)
    assert first_mismatch(to_np(K, "u64"), OK) is None


def test_merge_sort_full_size():
    """2**28 u64 keys uniform in [0, 2**24), payload = original index."""
    keys, vals = W.sort_input(DEV)
    src_k, src_v = keys.cpu().numpy().view(np.uint64), vals_np(vals)
    K, V, ws = tm.tm_merge_sort("u64", keys, vals)
    assert tm.tm_read_status(ws) == 0
    ck, cv = to_np(K, "u64"), vals_np(V)
    del K, V, keys, vals
    OK, OV = oracle.merge_sort(src_k, src_v, run=32)
    assert first_mismatch(ck, OK) is None
    assert first_mismatch(cv, OV) is None


def test_merge_sort_on_a_side_stream_with_binding_temporaries():
    """A call given a stream other than the current one makes its
    temporaries (tmp_keys, tmp_vals, workspace) on that stream: allocations
    of the same sizes on the current stream, filled at once while the sort
    still runs, cannot take their blocks."""
    n = 1 << 24
    g = torch.Generator().manual_seed(5)
    keys = torch.randint(0, 1 << 16, (n,), generator=g, dtype=torch.int64)
    vals = torch.arange(n, dtype=torch.int32)
    k, v = keys.to(DEV), vals.to(DEV)
    s = torch.cuda.Stream(DEV)
    s.wait_stream(torch.cuda.current_stream(DEV))
    K, V, ws = tm.tm_merge_sort("u64", k, v, stream=s)
    junk = [torch.full((n,), -1, dtype=torch.int64, device=DEV), torch.full((n,), -1, dtype=torch.int32, device=DEV)]
    torch.cuda.synchronize()
    assert tm.tm_read_status(ws) == 0
    OK, OV = oracle.merge_sort(to_np(keys, "u64"), vals_np(vals), run=32)
    assert first_mismatch(to_np(K, "u64"), OK) is None
    assert first_mismatch(vals_np(V), OV) is None
    del junk


DIGIT_CASES = ["top_byte", "full_64", "word_edge", "all_equal", "low_and_top", "u32_top"]


@pytest.mark.parametrize("case", DIGIT_CASES)
def test_run_formation_digit_windows(case):
    """The runs are sorted by 8-bit digits, skipping the bytes in which all
    keys of a run agree: keys that differ only in the top byte, in all 64
    bits, only in bits 31 and 32, nowhere, or in the lowest and the top byte
    (middle passes skipped); n spans three full runs of 4096 and a partial
    one.  The result is the oracle's stable sort."""
    n = 3 * 4096 + 17
    rng = np.random.default_rng(31 + DIGIT_CASES.index(case))
    if case == "top_byte":
        hk = rng.integers(0, 256, n, dtype=np.uint64) << np.uint64(56)
    elif case == "full_64":
        hk = rng.integers(0, 1 << 63, n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, n, dtype=np.uint64)
    elif case == "word_edge":
        hk = (rng.integers(0, 4, n, dtype=np.uint64) << np.uint64(31)) | np.uint64(0x5555)
    elif case == "all_equal":
        hk = np.full(n, 0x0123456789ABCDEF, dtype=np.uint64)
    elif case == "low_and_top":
        hk = (rng.integers(0, 4, n, dtype=np.uint64) << np.uint64(62)) | rng.integers(0, 3, n, dtype=np.uint64)
    else:
        hk = (rng.integers(0, 200, n, dtype=np.uint32) << np.uint32(24)).astype(np.uint32)
    kt = "u32" if case == "u32_top" else "u64"
    keys = torch.from_numpy(hk.view(np.int32) if kt == "u32" else hk.view(np.int64))
    vals = torch.arange(n, dtype=torch.int32)
    sort_check(keys, vals, kt)
    sort_check(keys, vals, kt, cfg={"merge_ways": 4})
