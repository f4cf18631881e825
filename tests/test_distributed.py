"""The distributed stable merge protocol (paper_1202_6575_gb300.distributed)
on the CPU: real gloo process groups of 2 and 4 ranks, and the thread
communicator with 1-5 ranks, the per-rank steps done by the oracle (rank
counts by its rank_low / rank_high, the plan by its five cases, the local
merge by its two-pointer merge).  Checked: the pieces of C, in rank order,
are the oracle's merge of the whole arrays; the segment bounds are points
of the merge path (chain points of the oracle's subproblems); the ranks
get equal shares of the subproblems; every exchanged segment is the
oracle's."""
import os
import threading

import numpy as np
import pytest
import torch

import oracle
from paper_1202_6575_gb300 import distributed as D


class OracleOps:
    """The protocol's per-rank steps by the oracle (test side only)."""

    def __init__(self, tile=64):
        self.tile = tile

    def blocks(self, n, m):
        return max(1, -(-(n + m) // self.tile))

    def rank(self, kind, q, X):
        f = oracle.rank_low if kind == "low" else oracle.rank_high
        x = X.numpy()
        return torch.tensor([f(v, x) for v in q.numpy()], dtype=torch.int64)

    def chain_points(self, n, m, p, xbar, ybar):
        t = oracle.subproblems(n, m, p, xbar.numpy(), ybar.numpy())
        pts = []
        for k in range(2 * p):
            if k < p and oracle.block_start(n, p, k) < n:
                pts.append((int(t[k, 0]), int(t[k, 2])))
            elif k >= p and oracle.block_start(m, p, k - p) < m:
                pts.append((int(t[k, 2]), int(t[k, 0])))
        pts.sort(key=lambda ab: (ab[0] + ab[1], ab[0]))
        return pts + [(n, m)]

    def sort(self, K, Kv):
        v = np.zeros(K.numel(), np.uint32) if Kv is None else Kv.numpy().view(np.uint32)
        k, sv = oracle.merge_sort(K.numpy(), v, run=32)
        return torch.from_numpy(k.copy()), (None if Kv is None else torch.from_numpy(sv.view(np.int32).copy()))

    def merge(self, A, Av, B, Bv):
        a, b = A.numpy(), B.numpy()
        if Av is None:
            K, _ = oracle.merge_two_pointer(a, np.zeros(len(a), np.uint32), b, np.zeros(len(b), np.uint32))
            return torch.from_numpy(K.copy()), None
        K, V = oracle.merge_two_pointer(a, Av.numpy().view(np.uint32), b, Bv.numpy().view(np.uint32))
        return torch.from_numpy(K.copy()), torch.from_numpy(V.view(np.int32).copy())


def make_case(seed, n, m, alphabet):
    g = torch.Generator().manual_seed(seed)
    A = torch.randint(0, alphabet, (n,), generator=g, dtype=torch.int32).sort().values
    B = torch.randint(0, alphabet, (m,), generator=g, dtype=torch.int32).sort().values
    Av = torch.arange(n, dtype=torch.int32)
    Bv = (torch.arange(m, dtype=torch.int64) | (1 << 31)).to(torch.int64)
    Bv = torch.where(Bv >= (1 << 31), Bv - (1 << 32), Bv).to(torch.int32)
    return A, Av, B, Bv


def cuts(total, G, seed):
    """G contiguous slices of uneven sizes (some empty)."""
    rng = np.random.default_rng(seed)
    c = sorted(int(v) for v in rng.integers(0, total + 1, G - 1))
    return [0] + c + [total]


def check(G, A, Av, B, Bv, results, keys_only=False):
    n, m = A.numel(), B.numel()
    K, V = oracle.merge_two_pointer(A.numpy(), Av.numpy().view(np.uint32), B.numpy(), Bv.numpy().view(np.uint32))
    # pieces in rank order, contiguous, the oracle's merge
    pos = 0
    for g in range(G):
        C, Cv, c_lo, plan = results[g]
        assert c_lo == pos
        assert np.array_equal(C.numpy(), K[pos:pos + C.numel()])
        if not keys_only:
            assert np.array_equal(Cv.numpy().view(np.uint32), V[pos:pos + C.numel()])
        pos += C.numel()
    assert pos == n + m
    # the bounds are merge-path points of the oracle's Steps 1-4, equal shares
    plan = results[0][3]
    p = plan["p"]
    xbar, ybar = oracle.cross_ranks(A.numpy(), B.numpy(), p)
    pts = OracleOps().chain_points(n, m, p, torch.from_numpy(xbar), torch.from_numpy(ybar))
    R = len(pts) - 1
    assert plan["records"] == R
    assert plan["bounds"] == [pts[(h * R) // G] for h in range(G)] + [(n, m)]
    for g in range(G):
        assert results[g][3]["bounds"] == plan["bounds"]


def run_threads(G, A, Av, B, Bv, ca, cb, keys_only=False):
    hub = D.ThreadHub(G)
    results = [None] * G
    errors = []

    def worker(g):
        try:
            results[g] = D.merge_distributed(A[ca[g]:ca[g + 1]], None if keys_only else Av[ca[g]:ca[g + 1]],
                                             B[cb[g]:cb[g + 1]], None if keys_only else Bv[cb[g]:cb[g + 1]],
                                             hub.comm(g), OracleOps())
        except Exception as e:                       # noqa: BLE001
            errors.append(e)
            hub.abort()

    ts = [threading.Thread(target=worker, args=(g,)) for g in range(G)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
    return results


@pytest.mark.parametrize("G", [1, 2, 3, 5])
@pytest.mark.parametrize("n,m,alphabet", [(0, 0, 5), (1, 0, 5), (0, 7, 5), (900, 600, 7), (1000, 3, 50),
                                          (4, 1200, 1000), (2000, 2000, 1), (3001, 1999, 100000)])
def test_thread_ranks_against_the_oracle(G, n, m, alphabet):
    A, Av, B, Bv = make_case(n * 7 + m + G, n, m, alphabet)
    ca, cb = cuts(n, G, n + G), cuts(m, G, m + 3 * G)
    check(G, A, Av, B, Bv, run_threads(G, A, Av, B, Bv, ca, cb))


def test_thread_ranks_keys_only():
    A, Av, B, Bv = make_case(1, 1500, 1100, 30)
    ca, cb = cuts(1500, 4, 1), cuts(1100, 4, 2)
    check(4, A, Av, B, Bv, run_threads(4, A, Av, B, Bv, ca, cb, keys_only=True), keys_only=True)


def _gloo_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A, Av, B, Bv = make_case(77 + world, 2500, 1800, 40)
        ca, cb = cuts(2500, world, 5 + world), cuts(1800, world, 9 + world)
        res = D.merge_distributed(A[ca[rank]:ca[rank + 1]], Av[ca[rank]:ca[rank + 1]],
                                  B[cb[rank]:cb[rank + 1]], Bv[cb[rank]:cb[rank + 1]],
                                  D.TorchComm(), OracleOps())
        torch.save(res, os.path.join(out_dir, f"r{rank}.pt"))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_process_groups(world, tmp_path):
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_gloo_worker, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    results = [torch.load(os.path.join(tmp_path, f"r{g}.pt"), weights_only=False) for g in range(world)]
    A, Av, B, Bv = make_case(77 + world, 2500, 1800, 40)
    check(world, A, Av, B, Bv, results)


def sort_case(seed, total, alphabet, G):
    g = torch.Generator().manual_seed(seed)
    K = torch.randint(0, alphabet, (total,), generator=g, dtype=torch.int32)
    Kv = torch.arange(total, dtype=torch.int32)
    return K, Kv, cuts(total, G, seed + 1)


def check_sort(G, K, Kv, results, keys_only=False):
    OK, OV = oracle.merge_sort(K.numpy(), Kv.numpy().view(np.uint32), run=1)
    pos = 0
    for g in range(G):
        C, Cv, c_lo = results[g]
        assert c_lo == pos
        assert np.array_equal(C.numpy(), OK[pos:pos + C.numel()])
        if not keys_only:
            assert np.array_equal(Cv.numpy().view(np.uint32), OV[pos:pos + C.numel()])
        pos += C.numel()
    assert pos == K.numel()


def run_sort_threads(G, K, Kv, cuts_, keys_only=False):
    hub = D.ThreadHub(G)
    results, errors = [None] * G, []

    def worker(g):
        try:
            results[g] = D.sort_distributed(K[cuts_[g]:cuts_[g + 1]],
                                            None if keys_only else Kv[cuts_[g]:cuts_[g + 1]],
                                            hub.comm(g), OracleOps())
        except Exception as e:                       # noqa: BLE001
            errors.append(e)
            hub.abort()

    ts = [threading.Thread(target=worker, args=(g,)) for g in range(G)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
    return results


@pytest.mark.parametrize("G", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("total,alphabet", [(0, 3), (1, 3), (5000, 7), (12001, 100000), (3000, 1)])
def test_sort_thread_ranks_against_the_oracle(G, total, alphabet):
    """Every rank's slice sorted locally, then rounds of distributed merges
    of neighbouring groups (G not a power of two leaves a group without a
    right half in some rounds); the pieces in rank order are the oracle's
    stable sort of the whole array, equal keys in their global order."""
    K, Kv, c = sort_case(total * 3 + G + alphabet, total, alphabet, G)
    check_sort(G, K, Kv, run_sort_threads(G, K, Kv, c))


def test_sort_thread_ranks_keys_only():
    K, Kv, c = sort_case(4, 7000, 50, 4)
    check_sort(4, K, Kv, run_sort_threads(4, K, Kv, c, keys_only=True), keys_only=True)


def _gloo_sort_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        K, Kv, c = sort_case(91 + world, 6000, 300, world)
        res = D.sort_distributed(K[c[rank]:c[rank + 1]], Kv[c[rank]:c[rank + 1]], D.TorchComm(), OracleOps())
        torch.save(res, os.path.join(out_dir, f"s{rank}.pt"))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_sort_gloo_process_groups(world, tmp_path):
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_gloo_sort_worker, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    results = [torch.load(os.path.join(tmp_path, f"s{g}.pt"), weights_only=False) for g in range(world)]
    K, Kv, _ = sort_case(91 + world, 6000, 300, world)
    check_sort(world, K, Kv, results)
