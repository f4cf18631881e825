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


# ---------------------------------------------------------------------------
# The value distributions match the stated recipe (statistical pins: each
# bound is several standard errors wide for the sample drawn)
# ---------------------------------------------------------------------------

def test_zipf_frequencies():
    # P(v) proportional to (v + 1)^-1.2 over 2^20 values: P(0) = 1 / H, with
    # H the generalised harmonic number (about 0.19), P(1) / P(0) = 2^-1.2
    N = 1 << 18
    x = W.large_merge("zipf", False, "cpu", log2n=18)[0].numpy()
    H = np.sum(np.arange(1, (1 << 20) + 1, dtype=np.float64) ** -1.2)
    p0 = 1.0 / H
    f0, f1 = np.mean(x == 0), np.mean(x == 1)
    assert 0.18 < p0 < 0.20
    assert abs(f0 - p0) < 5 * np.sqrt(p0 * (1 - p0) / N)
    p1 = p0 * 2.0 ** -1.2
    assert abs(f1 - p1) < 5 * np.sqrt(p1 * (1 - p1) / N)
    assert x.min() >= 0 and x.max() < (1 << 20)


def test_uniform_distributions():
    N = 1 << 18
    u = W.large_merge("uniform_1024", False, "cpu", log2n=18)[0].numpy()
    counts = np.bincount(u, minlength=1024)
    assert len(counts) == 1024 and abs(u.mean() - 511.5) < 5 * 295.6 / np.sqrt(N)
    assert counts.min() > 0.5 * N / 1024 and counts.max() < 1.5 * N / 1024
    f = W.large_merge("uniform_full", False, "cpu", log2n=18)[0].numpy().astype(np.float64)
    assert abs(f.mean()) < 5 * (2.0 ** 32 / np.sqrt(12)) / np.sqrt(N)
    assert f.min() < -(1 << 30) and f.max() > (1 << 30)
    k, v = W.sort_input("cpu", n=N)
    k = k.numpy().astype(np.float64)
    assert abs(k.mean() - (2 ** 24 - 1) / 2) < 5 * (2.0 ** 24 / np.sqrt(12)) / np.sqrt(N)
    assert k.min() >= 0 and k.max() < 2 ** 24 and v.numpy().tolist()[:3] == [0, 1, 2]


def test_one_million_merge_shape():
    A, Av, B, Bv = W.single_merge_1m("cpu")
    a, b = A.numpy(), B.numpy()
    assert len(a) == 1 << 20 and len(b) == 1 << 19
    assert a.min() >= 0 and a.max() < (1 << 16) and np.all(a[1:] >= a[:-1]) and np.all(b[1:] >= b[:-1])
    assert abs(len(a) / len(np.unique(a)) - 16) < 0.5                  # about 16 copies per value in A


def test_log_uniform_pair_lengths():
    # n_k = floor(2^(16 U)): half of the lengths lie below 2^8, a quarter below 2^4
    a_off, A, Av, b_off, B, Bv = W.batched_pairs("cpu", pairs=8192, log2_max=16)
    la = np.diff(a_off.numpy())
    lb = np.diff(b_off.numpy())
    for L in (la, lb):
        assert L.min() >= 1 and L.max() < (1 << 16)
        se = np.sqrt(0.25 / len(L))
        assert abs(np.mean(L < 256) - 0.5) < 5 * se and abs(np.mean(L < 16) - 0.25) < 5 * se
    assert np.corrcoef(la, lb)[0, 1] < 0.05                             # independent per side


def test_lsm_mixture():
    # log x is an equal mixture of N(0, 0.5^2), N(2, 0.5^2), N(5, 0.5^2)
    N = 1 << 18
    x = np.log(W.lsm_base("cpu", n=N)[0].numpy().astype(np.float64))
    assert abs(x.mean() - 7.0 / 3.0) < 0.02
    # a third of the mass in each component: split points 1 and 3.5 lie 2 and
    # 3 standard deviations from the neighbouring means
    lo, mid = np.mean(x < 1.0), np.mean((x >= 1.0) & (x < 3.5))
    assert abs(lo - 1 / 3) < 0.01 and abs(mid - 1 / 3) < 0.01


def test_widened_payloads_are_a_bijection_of_the_32_bit_tags():
    import numpy as np
    w = torch.tensor([0, 1, -1, 2**31 - 1, -2**31, 12345], dtype=torch.int32)
    v = W.widen_payload(w).numpy().view(np.uint64)
    t = w.numpy().view(np.uint32).astype(np.uint64)
    assert np.array_equal(v >> np.uint64(32), t)
    assert np.array_equal(v & np.uint64(0xFFFFFFFF), (t * np.uint64(0x9E3779B1)) & np.uint64(0xFFFFFFFF))
    assert len(set(v.tolist())) == len(v)
