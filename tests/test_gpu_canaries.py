"""Guard bands around every output: each form writes exactly its output
range (bulk-copy stores of the aligned middle, plain stores of the ragged
ends) and nothing beside it.  Outputs are sub-views of larger buffers filled
with a canary word; after the call the canaries must be intact and the
output must equal the oracle's."""
import numpy as np
import pytest
import torch

import oracle
from paper_1202_6575_gb300 import tm, workloads as W
from tests.helpers import first_mismatch, to_np, vals_np

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GUARD = 67                     # odd: the output starts at every alignment in turn
CANARY = -0x21524111           # 0xDEADBEEF as int32


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def guarded(count, dtype, shift):
    buf = torch.full((count + 2 * GUARD + shift,), CANARY, dtype=dtype, device=DEV)
    return buf, buf[GUARD + shift:GUARD + shift + count]


def intact(buf, shift, count):
    h = buf.cpu()
    return bool((h[:GUARD + shift] == CANARY).all()) and bool((h[GUARD + shift + count:] == CANARY).all())


@pytest.mark.parametrize("shift", [0, 1, 2, 3])
@pytest.mark.parametrize("kt,n,m,cfg", [("u32", 3001, 2000, {"p": 8}),                 # fused launch
                                        ("i32", 100003, 77777, None),                   # separate launches
                                        ("u64", 20001, 30007, {"tile": 512, "unfused": 1}),
                                        ("f32", 50000, 123, {"tile": 1024, "partition": 1})])
def test_merge_writes_only_its_output(kt, n, m, cfg, shift):
    A, Av, B, Bv = W.small_merge(n, m, kt, seed=n + m + shift, alphabet=500)
    kdt = {"u32": torch.int32, "i32": torch.int32, "u64": torch.int64, "f32": torch.float32}[kt]
    cbuf, C = guarded(n + m, kdt if kt != "f32" else torch.int32, shift)
    if kt == "f32":
        C = C.view(torch.float32)
    vbuf, Cv = guarded(n + m, torch.int32, shift)
    _, _, ws = tm.tm_merge(kt, A.to(DEV), Av.to(DEV), B.to(DEV), Bv.to(DEV), C, Cv, cfg=cfg)
    assert tm.tm_read_status(ws) == 0
    assert intact(cbuf, shift, n + m) and intact(vbuf, shift, n + m)
    K, V = oracle.merge_two_pointer(to_np(A, kt), vals_np(Av), to_np(B, kt), vals_np(Bv))
    assert first_mismatch(to_np(C, kt), K) is None and first_mismatch(vals_np(Cv), V) is None


@pytest.mark.parametrize("shift", [0, 3])
def test_keys_only_merge_writes_only_its_output(shift):
    A, Av, B, Bv = W.small_merge(40001, 30003, "u32", seed=shift, alphabet=100)
    cbuf, C = guarded(70004, torch.int32, shift)
    _, _, ws = tm.tm_merge("u32", A.to(DEV), None, B.to(DEV), None, C, None)
    assert tm.tm_read_status(ws) == 0 and intact(cbuf, shift, 70004)
    K, _ = oracle.merge_two_pointer(to_np(A, "u32"), vals_np(Av), to_np(B, "u32"), vals_np(Bv))
    assert first_mismatch(to_np(C, "u32"), K) is None


@pytest.mark.parametrize("shift", [0, 1])
def test_batched_and_sort_write_only_their_output(shift):
    a_off, A, Av, b_off, B, Bv = W.batched_pairs("cpu", pairs=500, log2_max=12, seed=41)
    total = A.numel() + B.numel()
    cbuf, C = guarded(total, torch.int64, shift)
    vbuf, Cv = guarded(total, torch.int32, shift)
    d = lambda t: t.to(DEV)
    _, _, ws = tm.tm_merge_batched("u64", d(a_off), d(A), d(Av), d(b_off), d(B), d(Bv), C, Cv)
    assert tm.tm_read_status(ws) == 0 and intact(cbuf, shift, total) and intact(vbuf, shift, total)
    K, V = oracle.merge_batched(a_off.numpy(), to_np(A, "u64"), vals_np(Av), b_off.numpy(), to_np(B, "u64"),
                                vals_np(Bv))
    assert first_mismatch(to_np(C, "u64"), K) is None and first_mismatch(vals_np(Cv), V) is None
    n = 100003
    keys, vals = W.sort_input("cpu", n=n, key_bits=10)
    kbuf, kk = guarded(n, torch.int64, shift)
    vb2, vv = guarded(n, torch.int32, shift)
    tkbuf, tk = guarded(n, torch.int64, shift)
    tvbuf, tv = guarded(n, torch.int32, shift)
    kk.copy_(keys.to(DEV))
    vv.copy_(vals.to(DEV))
    _, _, ws = tm.tm_merge_sort("u64", kk, vv, tk, tv)
    assert tm.tm_read_status(ws) == 0
    assert all(intact(b, shift, n) for b in (kbuf, vb2, tkbuf, tvbuf))
    OK, OV = oracle.merge_sort(to_np(keys, "u64"), vals_np(vals), run=32)
    assert first_mismatch(to_np(kk, "u64"), OK) is None and first_mismatch(vals_np(vv), OV) is None
