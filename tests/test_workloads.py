"""The seeded generators produce what the workloads describe (CPU, small sizes)."""
import numpy as np
import torch

from paper_1202_6575_gb300 import workloads as W


def u32(t):
    return t.numpy().view(np.uint32)


def test_payload_tags():
    v = u32(W.payload(1, 5, "cpu", start=3))
    assert v.tolist() == [(1 << 31) | k for k in range(3, 8)]
    assert u32(W.payload(0, 3, "cpu")).tolist() == [0, 1, 2]


def test_large_merge_shapes_small():
    for dist in W.DIST_NAMES:
        for skewed in (False, True):
            A, Av, B, Bv = W.large_merge(dist, skewed, "cpu", log2n=12, log2m_skewed=5)
            assert len(A) == 4096 and len(B) == (32 if skewed else 4096)
            for X in (A, B):
                x = X.numpy()
                assert np.all(x[1:] >= x[:-1]) and X.dtype == torch.int32
            if dist == "all_equal":
                assert int(A.abs().sum()) == 0
            if dist == "uniform_1024":
                assert int(A.min()) >= 0 and int(A.max()) < 1024


def test_determinism():
    a = W.large_merge("zipf", False, "cpu", log2n=10)[0]
    b = W.large_merge("zipf", False, "cpu", log2n=10)[0]
    assert torch.equal(a, b)


def test_batched_pairs_small():
    a_off, A, Av, b_off, B, Bv = W.batched_pairs("cpu", pairs=50, log2_max=8)
    assert a_off[0] == 0 and b_off[0] == 0 and len(a_off) == 51
    la = (a_off[1:] - a_off[:-1]).numpy()
    assert la.min() >= 1 and la.max() <= 256
    a = A.numpy()
    for k in range(50):
        seg = a[a_off[k]:a_off[k + 1]]
        assert np.all(seg[1:] >= seg[:-1]) and seg.min() >= 0 and seg.max() < (1 << 20)


def test_lsm_inputs_small():
    X, Xv = W.lsm_base("cpu", n=1000)
    Y, Yv = W.lsm_batch(3, "cpu", size=100, base_n=1000)
    x = X.numpy()
    assert x.dtype == np.float32 and np.all(x[1:] >= x[:-1]) and np.all(x > 0)
    assert Yv[0].item() == 1000 + 3 * 100
