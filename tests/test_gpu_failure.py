"""Failure detection without a GPU fault: a wait that runs out.

The persistent tile kernel's waits on its stage barriers are bounded.  With
the testing field `test_drop_tile` set, every CTA withholds the readiness
signal of one staged tile; its consumers' wait runs out after `wait_ms`, the
kernel records TM_ERR_TIMEOUT in the status word and returns.  The host
reads the status, and the context stays usable for the next call."""
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


def test_bounded_wait_reports_timeout_and_context_survives():
    A, Av, B, Bv = W.small_merge(1 << 22, 1 << 22, "u32", seed=9, alphabet=1 << 20)
    dA, dAv, dB, dBv = (t.to(DEV) for t in (A, Av, B, Bv))
    C, Cv, ws = tm.tm_merge("u32", dA, dAv, dB, dBv, cfg={"wait_ms": 200, "test_drop_tile": 2})
    assert tm.tm_read_status(ws) == tm.TM_ERR_TIMEOUT
    # the same merge without the withheld signal succeeds on the same context
    C, Cv, ws = tm.tm_merge("u32", dA, dAv, dB, dBv)
    assert tm.tm_read_status(ws) == 0
    K, V = oracle.merge_two_pointer(to_np(A, "u32"), vals_np(Av), to_np(B, "u32"), vals_np(Bv))
    assert first_mismatch(to_np(C, "u32"), K) is None and first_mismatch(vals_np(Cv), V) is None


def test_invalid_arguments_launch_nothing():
    A = torch.zeros(10, dtype=torch.int32, device=DEV)
    with pytest.raises(tm.TmError) as e:
        tm.tm_merge("u32", A, A, A, A, cfg={"threads": 96})     # not a supported thread count
    assert e.value.code in (tm.TM_ERR_UNSUPPORTED, tm.TM_ERR_INVALID)
