"""Segmented stable merge sort (tm_merge_sort_segmented): every segment
sorted stably and independently; compared with the oracle's stable merge
sort of each segment, bit for bit (keys and payloads = original index)."""
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


def check(keys, vals, offs, kt, cfg=None):
    hk = to_np(keys, kt)
    hv = None if vals is None else vals_np(vals)
    K, V, ws = tm.tm_merge_sort_segmented(kt, keys.to(DEV).clone(), None if vals is None else vals.to(DEV).clone(),
                                          offs, cfg=cfg)
    assert tm.tm_read_status(ws) == 0
    ck = to_np(K, kt)
    cv = None if V is None else vals_np(V)
    for q in range(len(offs) - 1):
        a, b = int(offs[q]), int(offs[q + 1])
        ok, ov = oracle.merge_sort(hk[a:b], np.arange(a, b, dtype=np.uint32) if hv is None else hv[a:b], run=32)
        assert first_mismatch(ck[a:b], ok) is None, f"keys of segment {q}"
        if cv is not None:
            assert first_mismatch(cv[a:b], ov) is None, f"payloads of segment {q}"


@pytest.mark.parametrize("kt", ["u32", "i32", "u64", "f32"])
def test_segment_length_mix(kt):
    lens = [0, 1, 2, 1023, 1024, 1025, 0, 2048, 4095, 4096, 4097, 8193, 5000, 3, 70000, 0, 1 << 17, 777]
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    n = int(offs[-1])
    g = torch.Generator().manual_seed(len(kt))
    keys = torch.randint(-500, 500, (n,), generator=g, dtype=torch.int64)
    keys = {"u64": keys + 500, "u32": (keys + 500).to(torch.int32), "i32": keys.to(torch.int32),
            "f32": (keys * 0.5).to(torch.float32)}[kt]
    vals = torch.arange(n, dtype=torch.int32)
    check(keys, vals, offs, kt)


def test_many_log_uniform_segments_tiles_and_payload_widths():
    g = torch.Generator().manual_seed(3)
    lens = torch.exp(torch.rand(3000, generator=g) * np.log(1 << 14)).long().tolist()
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    n = int(offs[-1])
    keys = torch.randint(0, 1 << 10, (n,), generator=g, dtype=torch.int64)
    vals = torch.arange(n, dtype=torch.int32)
    for cfg in (None, {"tile": 1024}, {"tile": 4096}):
        check(keys, vals, offs, "u64", cfg)
    check(keys, None, offs, "u64")                       # keys only
    # 8-byte payloads: the widened tags travel with the keys
    K, Vw, ws = tm.tm_merge_sort_segmented("u64", keys.to(DEV).clone(), W.widen_payload(vals).to(DEV), offs)
    assert tm.tm_read_status(ws) == 0
    hk = to_np(keys, "u64")
    tags = Vw.cpu().numpy().view(np.uint64) >> np.uint64(32)
    for q in range(0, len(offs) - 1, 97):
        a, b = int(offs[q]), int(offs[q + 1])
        ok, ov = oracle.merge_sort(hk[a:b], np.arange(a, b, dtype=np.uint32), run=32)
        assert first_mismatch(to_np(K, "u64")[a:b], ok) is None
        assert first_mismatch(tags[a:b], ov.astype(np.uint64)) is None


def test_one_segment_equals_the_plain_sort():
    keys, vals = W.sort_input("cpu", n=(1 << 20) + 17, key_bits=12)
    n = keys.numel()
    K1, V1, _ = tm.tm_merge_sort_segmented("u64", keys.to(DEV).clone(), vals.to(DEV).clone(), [0, n])
    K2, V2, _ = tm.tm_merge_sort("u64", keys.to(DEV).clone(), vals.to(DEV).clone())
    assert torch.equal(K1, K2) and torch.equal(V1, V2)
