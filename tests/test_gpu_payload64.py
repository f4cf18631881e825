"""GPU parity with 8-byte payload words (tm_config.payload_bytes = 8).

The oracle moves 32-bit payloads; a stable merge or sort moves every payload
with its key whatever its width, so the expected 64-bit output is the
oracle's output of the 32-bit source tags, each widened by the same
bijection the inputs were made with (workloads.widen_payload).  Keys and
payloads are compared bit-exactly."""
import numpy as np
import pytest
import torch

import oracle
from paper_1202_6575_gb300 import tm, workloads as W
from tests.helpers import to_np, vals_np, first_mismatch

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def wide_np(tags_u32: np.ndarray) -> np.ndarray:
    return W.widen_payload(torch.from_numpy(tags_u32.view(np.int32))).numpy().view(np.uint64)


def merge64_check(kt, n, m, cfg, seed, alphabet=300):
    A, Av, B, Bv = W.small_merge(n, m, kt, seed=seed, alphabet=alphabet)
    Aw, Bw = W.widen_payload(Av), W.widen_payload(Bv)
    C, Cw, ws = tm.tm_merge(kt, A.to(DEV), Aw.to(DEV), B.to(DEV), Bw.to(DEV), cfg=cfg)
    assert Cw.dtype == torch.int64
    assert tm.tm_read_status(ws) == 0
    K, V = oracle.merge_two_pointer(to_np(A, kt), vals_np(Av), to_np(B, kt), vals_np(Bv))
    assert first_mismatch(to_np(C, kt), K) is None, "keys"
    assert first_mismatch(Cw.cpu().numpy().view(np.uint64), wide_np(V)) is None, "payloads"


@pytest.mark.parametrize("kt", ["u32", "i32", "u64", "f32"])
@pytest.mark.parametrize("n,m,cfg", [(1, 0, None), (0, 7, None), (5000, 3001, {"p": 8}),
                                     (200003, 150001, None), (200003, 150001, {"unfused": 1}),
                                     (70001, 50003, {"tile": 4096, "threads": 256}),
                                     (30011, 20011, {"split": 1}), (30011, 20011, {"split": 1, "threads": 512}),
                                     (100003, 77777, {"partition": 1}),
                                     ((1 << 16) + 3, (1 << 15) - 1, {"p": 1024})])
def test_payload64_merges(kt, n, m, cfg):
    merge64_check(kt, n, m, cfg, seed=n + 3 * m + 17)


@pytest.mark.parametrize("kt", ["u32", "u64"])
def test_payload64_merge_beyond_the_fused_range(kt):
    """Above the fused launch's range the default merge of 8-byte payloads
    runs 256 consumer threads; every key and payload equals the oracle's."""
    merge64_check(kt, (1 << 25) + 5, 1 << 24, None, seed=3, alphabet=None)


@pytest.mark.parametrize("kt", ["u32", "u64"])
def test_payload64_batched(kt):
    g = torch.Generator().manual_seed(5)
    pairs = 3000
    la = torch.randint(0, 300, (pairs,), generator=g)
    lb = torch.randint(0, 300, (pairs,), generator=g)
    la[::7] = 0
    a_off = torch.cat([torch.zeros(1, dtype=torch.int64), torch.cumsum(la, 0)])
    b_off = torch.cat([torch.zeros(1, dtype=torch.int64), torch.cumsum(lb, 0)])
    ta, tb = int(a_off[-1]), int(b_off[-1])
    dt = torch.int64 if kt == "u64" else torch.int32
    seg_a = torch.repeat_interleave(torch.arange(pairs), la)
    seg_b = torch.repeat_interleave(torch.arange(pairs), lb)
    # keys sorted within each pair: sort by (pair, key)
    ka = torch.randint(0, 50, (ta,), generator=g)
    kb = torch.randint(0, 50, (tb,), generator=g)
    A = (seg_a * 64 + ka).sort().values % 64 if ta else ka
    B = (seg_b * 64 + kb).sort().values % 64 if tb else kb
    A, B = A.to(dt), B.to(dt)
    Av, Bv = W.payload(0, ta, "cpu"), W.payload(1, tb, "cpu")
    C, Cw, ws = tm.tm_merge_batched(kt, a_off.to(DEV), A.to(DEV), W.widen_payload(Av).to(DEV), b_off.to(DEV),
                                    B.to(DEV), W.widen_payload(Bv).to(DEV))
    assert tm.tm_read_status(ws) == 0
    K, V = oracle.merge_batched(a_off.numpy(), to_np(A, kt), vals_np(Av), b_off.numpy(), to_np(B, kt), vals_np(Bv))
    assert first_mismatch(to_np(C, kt), K) is None
    assert first_mismatch(Cw.cpu().numpy().view(np.uint64), wide_np(V)) is None


@pytest.mark.parametrize("n", [0, 1, 1000, 1025, 5000, 65537, (1 << 20) + 3])
def test_payload64_sort(n):
    g = torch.Generator().manual_seed(n + 1)
    keys = torch.randint(0, 1 << 12, (n,), generator=g, dtype=torch.int64)
    tags = W.payload(0, n, "cpu")
    OK, OV = oracle.merge_sort(to_np(keys, "u64"), vals_np(tags), run=32)
    for cfg in (None, {"merge_ways": 4}):
        K, Vw, ws = tm.tm_merge_sort("u64", keys.to(DEV).clone(), W.widen_payload(tags).to(DEV), cfg=cfg)
        assert tm.tm_read_status(ws) == 0
        assert first_mismatch(to_np(K, "u64"), OK) is None
        assert first_mismatch(Vw.cpu().numpy().view(np.uint64), wide_np(OV)) is None


def test_payload64_large_merge_full_size():
    """n = m = 2**28 int32 keys (uniform over int32) with 8-byte payloads, the
    default launch configuration; every output element compared."""
    A, Av, B, Bv = W.large_merge("uniform_full", False, DEV)
    Aw, Bw = W.widen_payload(Av), W.widen_payload(Bv)
    hA, hAv, hB, hBv = to_np(A, "i32"), vals_np(Av), to_np(B, "i32"), vals_np(Bv)
    del Av, Bv
    C, Cw, ws = tm.tm_merge("i32", A, Aw, B, Bw)
    assert tm.tm_read_status(ws) == 0
    del A, Aw, B, Bw
    ck, cw = to_np(C, "i32"), Cw.cpu().numpy().view(np.uint64)
    del C, Cw
    torch.cuda.empty_cache()
    K, V = oracle.merge_two_pointer(hA, hAv, hB, hBv)
    assert first_mismatch(ck, K) is None
    assert first_mismatch(cw >> np.uint64(32), V.astype(np.uint64)) is None, "high words (the tags)"
    assert first_mismatch(cw, wide_np(V)) is None, "low words"


def test_payload64_sort_full_size():
    """2**28 u64 keys uniform in [0, 2**24) with 8-byte payloads; checked
    against the oracle's stable sort of the 32-bit tags."""
    keys, tags = W.sort_input(DEV)
    src_k, src_t = keys.cpu().numpy().view(np.uint64), vals_np(tags)
    K, Vw, ws = tm.tm_merge_sort("u64", keys, W.widen_payload(tags))
    assert tm.tm_read_status(ws) == 0
    ck, cw = to_np(K, "u64"), Vw.cpu().numpy().view(np.uint64)
    del K, Vw, keys, tags
    torch.cuda.empty_cache()
    OK, OV = oracle.merge_sort(src_k, src_t, run=32)
    assert first_mismatch(ck, OK) is None
    assert first_mismatch(cw >> np.uint64(32), OV.astype(np.uint64)) is None
    assert first_mismatch(cw, wide_np(OV)) is None
