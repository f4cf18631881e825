"""The learned merge on the full LSM workload: a sorted float32 base of 2^28
keys (three lognormals, payload = insertion number) merged 256 times with
sorted batches of 2^20 keys of the same mixture, the base on the A side and
the model's knot ranks advanced by every merge (base' = merge(base, batch)).
Every merge's cross ranks, the learned ones (the B-block starts searched in
the base) included, equal the plain search's (all 256 merges); the merged
base equals the oracle's two-pointer merge on the first merge, every 16th
and the last (17 of the 256: the oracle's CPU merge of a 2^28-element base
is the slow part); the model falls back to the full search on at most 1 %
of its searches."""
import pytest
import torch

import oracle
from paper_1202_6575_gb300 import tm, workloads as W
from tests.helpers import first_mismatch, vals_np

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_lsm_256_merges_of_2p20_into_2p28():
    N0, m, merges = 1 << 28, 1 << 20, 256
    cap = N0 + merges * m
    X0, X0v = W.lsm_base(DEV, n=N0)
    q = W.lsm_label_keys(DEV, count=1 << 18)
    init = W.cdf_init(hidden=64)
    flat = torch.cat([init["W1"].reshape(-1), init["b1"], init["w2"], init["b2"].reshape(1)])
    model = tm.CdfModel(4096, 64, DEV).init(X0, flat)
    model.train(q, tm.tm_rank_search("f32", "high", q, X0), steps=400, lr=3e-3)
    qc = W.lsm_label_keys(DEV, count=1 << 20, seed=W.SEED_BASE + 8)
    model.calibrate(qc, tm.tm_rank_search("f32", "high", qc, X0))

    bufs = [(torch.empty(cap, dtype=torch.float32, device=DEV), torch.empty(cap, dtype=torch.int32, device=DEV))
            for _ in range(2)]
    bufs[0][0][:N0].copy_(X0)
    bufs[0][1][:N0].copy_(X0v)
    del X0, X0v, q, qc
    ws = tm.new_workspace(tm.tm_merge_workspace_size(cap - m, m), DEV)
    checked = {0, merges - 1} | set(range(15, merges, 16))
    n, src = N0, 0
    for k in range(merges):
        A, Av = bufs[src][0][:n], bufs[src][1][:n]
        B, Bv = W.lsm_batch(k, DEV, size=m, base_n=N0)
        C, Cv = bufs[src ^ 1][0][:n + m], bufs[src ^ 1][1][:n + m]
        p = tm.tm_merge_blocks(n, m)
        xp, yp = tm.tm_cross_ranks("f32", A, B, p)
        tm.tm_merge_learned(model, A, Av, B, Bv, C, Cv, ws, flags=tm.LEARNED_ADVANCE)
        assert tm.tm_read_status(ws) == 0, k
        # the workspace holds the learned call's cross ranks: xbar after the
        # 256-byte control block, ybar on the next 256-byte boundary
        y_off = 256 + (8 * (p + 1) + 255) // 256 * 256
        xl = ws[256:256 + 8 * (p + 1)].view(torch.int64)
        yl = ws[y_off:y_off + 8 * (p + 1)].view(torch.int64)
        assert torch.equal(xl, xp) and torch.equal(yl, yp), k
        if k in checked:
            K, V = oracle.merge_two_pointer(A.cpu().numpy(), vals_np(Av), B.cpu().numpy(), vals_np(Bv))
            assert first_mismatch(C.cpu().numpy(), K) is None, k
            assert first_mismatch(vals_np(Cv), V) is None, k
            del K, V
        n += m
        src ^= 1
    h = model.header()
    assert h["N"] == cap and n == cap
    assert h["learned"] > 0 and h["fallbacks"] <= 0.01 * h["learned"], (h["fallbacks"], h["learned"])
