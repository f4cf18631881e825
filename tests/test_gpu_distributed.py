"""The distributed stable merge protocol with the library's kernels doing
every rank's steps (rank searches, the plan, the local tm_merge), the ranks
as threads of one process exchanging through ThreadComm (the collectives
are host-side, so no kernel waits on another).  The pieces of C, in rank
order, are compared with the oracle's merge of the whole arrays, bit for
bit."""
import threading

import numpy as np
import pytest
import torch

import oracle
from paper_1202_6575_gb300 import distributed as D, tm, workloads as W
from tests.helpers import to_np, vals_np

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    tm.load()


def run(G, kt, A, Av, B, Bv, ca, cb, cfg=None):
    hub = D.ThreadHub(G)
    results, errors = [None] * G, []

    def worker(g):
        try:
            torch.cuda.set_device(0)
            sl = lambda t, c: None if t is None else t[c[g]:c[g + 1]]
            results[g] = D.merge_distributed(sl(A, ca), sl(Av, ca), sl(B, cb), sl(Bv, cb), hub.comm(g),
                                             D.GpuOps(kt, cfg))
        except Exception as e:                       # noqa: BLE001
            errors.append(e)
            hub.abort()

    ts = [threading.Thread(target=worker, args=(g,)) for g in range(G)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
    torch.cuda.synchronize()
    return results


@pytest.mark.parametrize("G", [1, 2, 3, 4])
@pytest.mark.parametrize("kt,n,m,cfg", [("u32", 1 << 20, 1 << 19, None), ("i32", 300001, 5, {"tile": 1024}),
                                        ("u64", 77777, 250003, None), ("f32", 0, 4097, None)])
def test_distributed_merge_threads_against_the_oracle(G, kt, n, m, cfg):
    A, Av, B, Bv = W.small_merge(n, m, kt, seed=n + m + G, alphabet=5000)
    rng = np.random.default_rng(G + n)
    ca = [0] + sorted(int(v) for v in rng.integers(0, n + 1, G - 1)) + [n]
    cb = [0] + sorted(int(v) for v in rng.integers(0, m + 1, G - 1)) + [m]
    d = [t.to(DEV) for t in (A, Av, B, Bv)]
    results = run(G, kt, *d, ca, cb, cfg)
    K, V = oracle.merge_two_pointer(to_np(A, kt), vals_np(Av), to_np(B, kt), vals_np(Bv))
    pos = 0
    for g in range(G):
        C, Cv, c_lo, plan = results[g]
        assert c_lo == pos
        assert np.array_equal(to_np(C, kt), K[pos:pos + C.numel()])
        assert np.array_equal(vals_np(Cv), V[pos:pos + C.numel()])
        pos += C.numel()
    assert pos == n + m
    # every rank got an equal share of the subproblems
    R = results[0][3]["records"]
    assert R == tm.tm_plan_tile_count(n, m, results[0][3]["p"])


def test_distributed_merge_keys_only_and_wide_payloads():
    n, m, G = 200003, 150001, 3
    A, Av, B, Bv = W.small_merge(n, m, "u32", seed=5, alphabet=100)
    ca, cb = [0, 1000, 150000, n], [0, 0, 90000, m]
    K, V = oracle.merge_two_pointer(to_np(A, "u32"), vals_np(Av), to_np(B, "u32"), vals_np(Bv))
    res = run(G, "u32", A.to(DEV), None, B.to(DEV), None, ca, cb)
    assert np.array_equal(np.concatenate([to_np(r[0], "u32") for r in res]), K)
    Aw, Bw = W.widen_payload(Av).to(DEV), W.widen_payload(Bv).to(DEV)
    res = run(G, "u32", A.to(DEV), Aw, B.to(DEV), Bw, ca, cb)
    got = np.concatenate([r[1].cpu().numpy().view(np.uint64) for r in res])
    assert np.array_equal(got >> np.uint64(32), V.astype(np.uint64))


def run_sort(G, kt, K, Kv, c, cfg=None):
    hub = D.ThreadHub(G)
    results, errors = [None] * G, []

    def worker(g):
        try:
            torch.cuda.set_device(0)
            results[g] = D.sort_distributed(K[c[g]:c[g + 1]], None if Kv is None else Kv[c[g]:c[g + 1]],
                                            hub.comm(g), D.GpuOps(kt, cfg))
        except Exception as e:                       # noqa: BLE001
            errors.append(e)
            hub.abort()

    ts = [threading.Thread(target=worker, args=(g,)) for g in range(G)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
    torch.cuda.synchronize()
    return results


@pytest.mark.parametrize("G", [1, 2, 3, 4])
@pytest.mark.parametrize("kt,total", [("u64", 300007), ("i32", 99991), ("f32", 4096 * 5 + 1), ("u32", 0)])
def test_distributed_sort_threads_against_the_oracle(G, kt, total):
    """Local tm_merge_sort of every rank's slice, then distributed merges of
    neighbouring groups of ranks; the pieces in rank order are the oracle's
    stable sort of the whole array."""
    g = torch.Generator().manual_seed(total + G)
    raw = torch.randint(-3000, 3000, (total,), generator=g, dtype=torch.int64)
    K = {"u64": raw + 3000, "i32": raw.to(torch.int32), "f32": (raw * 0.5).to(torch.float32),
         "u32": raw.to(torch.int32)}[kt]
    Kv = W.payload(0, total, "cpu")
    rng = np.random.default_rng(G + total)
    c = [0] + sorted(int(v) for v in rng.integers(0, total + 1, G - 1)) + [total]
    res = run_sort(G, kt, K.to(DEV), Kv.to(DEV), c)
    OK, OV = oracle.merge_sort(to_np(K, kt), vals_np(Kv), run=1)
    pos = 0
    for r in range(G):
        C, Cv, c_lo = res[r]
        assert c_lo == pos
        assert np.array_equal(to_np(C, kt), OK[pos:pos + C.numel()])
        assert np.array_equal(vals_np(Cv), OV[pos:pos + C.numel()])
        pos += C.numel()
    assert pos == total


def test_distributed_sort_keys_only():
    total, G = 50000, 3
    g = torch.Generator().manual_seed(1)
    K = torch.randint(0, 77, (total,), generator=g, dtype=torch.int64)
    res = run_sort(G, "u64", K.to(DEV), None, [0, 20000, 20000, total])
    got = np.concatenate([to_np(r[0], "u64") for r in res])
    assert np.array_equal(got, np.sort(to_np(K, "u64"), kind="stable"))
