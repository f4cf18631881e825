"""tm_merge_noalloc: the merge entry point that allocates nothing.

Some callers cannot allocate device memory or hand the library a workspace
(code hosted by a framework that passes it only input and output buffers,
loops that must never hit the allocator).  tm_merge_noalloc keeps its cross
ranks in a device array built into the library instead.  These tests call it
through the C ABI and check it against tm_merge and against the CPU oracle's
two-pointer stable merge, bit for bit, on two calls in a row (the second call
reuses the array the first one left behind).  The file is named so that
pytest collects it last.
"""
import numpy as np
import pytest
import torch

import oracle
from tests.helpers import NP_KEY, vals_np
from paper_1202_6575_gb300 import tm, workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _inputs(n, m, kt, seed):
    A, Av, B, Bv = W.small_merge(n, m, kt, seed=seed, alphabet=1000)
    return A.to(DEV), Av.to(DEV), B.to(DEV), Bv.to(DEV)


@pytest.mark.parametrize("kt,cfg", [("u32", None), ("u64", {"tile": 1024}), ("i32", {"p": 1024})])
def test_noalloc_matches_tm_merge_on_two_calls_in_a_row(kt, cfg):
    # a large call, then a smaller one that leaves stale entries of the first
    for n, m, seed in ((300000, 200003, 11), (70001, 5, 12)):
        A, Av, B, Bv = _inputs(n, m, kt, seed)
        C_ref, Cv_ref, ws = tm.tm_merge(kt, A, Av, B, Bv, cfg=cfg)
        assert tm.tm_read_status(ws) == 0
        C = torch.full_like(C_ref, -7)
        Cv = torch.full_like(Cv_ref, -7)
        status = torch.full((1,), -1, dtype=torch.int32, device=DEV)   # the call must clear it
        tm.tm_merge_noalloc(kt, A, Av, B, Bv, C, Cv, status, cfg=cfg)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(C, C_ref)
        assert torch.equal(Cv, Cv_ref)
        K, V = oracle.merge_two_pointer(A.cpu().numpy().view(NP_KEY[kt]), vals_np(Av),
                                        B.cpu().numpy().view(NP_KEY[kt]), vals_np(Bv))
        assert np.array_equal(C.cpu().numpy().view(NP_KEY[kt]), K)
        assert np.array_equal(vals_np(Cv), V)


def test_noalloc_rejects_more_blocks_than_its_array_holds():
    A, Av, B, Bv = _inputs(1000, 1000, "u32", 3)
    C = torch.empty(2000, dtype=torch.int32, device=DEV)
    Cv = torch.empty(2000, dtype=torch.int32, device=DEV)
    with pytest.raises(tm.TmError) as e:
        tm.tm_merge_noalloc("u32", A, Av, B, Bv, C, Cv, cfg={"p": 262144})
    assert e.value.code == tm.TM_ERR_WORKSPACE
    tm.tm_merge_noalloc("u32", A, Av, B, Bv, C, Cv, cfg={"p": 262143})   # the largest accepted
    C_ref, Cv_ref, _ = tm.tm_merge("u32", A, Av, B, Bv, cfg={"p": 262143})
    torch.cuda.synchronize()
    assert torch.equal(C, C_ref) and torch.equal(Cv, Cv_ref)
