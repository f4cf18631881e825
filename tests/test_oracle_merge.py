"""Pins of the merge oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: the values
printed in Figure 1, Python's own stable sort (a library routine), brute-force
counting, closed forms and invariants.  No GPU is used.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "figure1.json")
DTYPES = [np.uint32, np.int32, np.uint64, np.float32]


def tag(src, idx):
    return (src << 31) | idx


def stable_reference(A, B):
    """Stable sort of the tagged concatenation A||B by key alone (Python's
    sorted() is stable): the unique stable merge of Section 2."""
    items = [(A[i], tag(0, i)) for i in range(len(A))] + [(B[j], tag(1, j)) for j in range(len(B))]
    items = sorted(items, key=lambda t: t[0])
    keys = np.array([k for k, _ in items], dtype=A.dtype)
    vals = np.array([v for _, v in items], dtype=np.uint32)
    return keys, vals


def payloads(n, m):
    return (np.arange(n, dtype=np.uint32),
            (np.arange(m, dtype=np.uint64) | (1 << 31)).astype(np.uint32))


def rand_sorted(rng, n, dtype, alphabet):
    x = np.sort(rng.integers(0, alphabet, size=n))
    if dtype == np.float32:
        return (x * 0.25 - 3.0).astype(np.float32)
    if dtype == np.int32:
        return (x - alphabet // 2).astype(np.int32)
    return x.astype(dtype)


# ---------------------------------------------------------------------------
# Figure 1 (Section 2), the paper's worked example
# ---------------------------------------------------------------------------

def load_golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_figure1_block_starts():
    g = load_golden()
    n, m, p = len(g["A"]), len(g["B"]), g["p"]
    assert [oracle.block_start(n, p, i) for i in range(p + 1)] == g["x"]
    assert [oracle.block_start(m, p, j) for j in range(p + 1)] == g["y"]


def test_figure1_cross_ranks():
    g = load_golden()
    A = np.array(g["A"], dtype=np.uint32)
    B = np.array(g["B"], dtype=np.uint32)
    xbar, ybar = oracle.cross_ranks(A, B, g["p"])
    assert xbar.tolist() == g["xbar"]
    assert ybar.tolist() == g["ybar"]


@pytest.mark.parametrize("dtype", DTYPES)
def test_figure1_subproblems(dtype):
    g = load_golden()
    A = np.array(g["A"], dtype=dtype)
    B = np.array(g["B"], dtype=dtype)
    p = g["p"]
    Av, Bv = payloads(len(A), len(B))
    C, Cv, xbar, ybar, table = oracle.paper_merge(A, Av, B, Bv, p)

    def rng_of(pair):
        return (0, 0) if pair is None else (pair[0], pair[1] + 1)

    for row, exp in zip(table[:p], g["step3"]):
        lo, hi, olo, ohi, c0, case = row
        a = rng_of(exp["A"])
        b = rng_of(exp["B"])
        assert (lo, hi) == a
        if exp["B"] is None:
            assert olo == ohi
        else:
            assert (olo, ohi) == b
        assert c0 == exp["C"][0]
        assert c0 + (hi - lo) + (ohi - olo) == exp["C"][1] + 1
        if exp["case"]:
            assert chr(case) == exp["case"]
    for row, exp in zip(table[p:], g["step4"]):
        lo, hi, olo, ohi, c0, case = row
        assert (lo, hi) == rng_of(exp["B"])
        if exp["A"] is None:
            assert olo == ohi
        else:
            assert (olo, ohi) == rng_of(exp["A"])
        assert c0 == exp["C"][0]
        assert c0 + (hi - lo) + (ohi - olo) == exp["C"][1] + 1
        if exp["case"]:
            assert chr(case) == exp["case"]
    K, V = stable_reference(A, B)
    assert np.array_equal(C, K) and np.array_equal(Cv, V)


# ---------------------------------------------------------------------------
# Rank primitives (Section 2 definitions) against brute-force counting
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", DTYPES)
def test_ranks_against_counting(dtype):
    rng = np.random.default_rng(11)
    for length in [0, 1, 2, 3, 7, 16, 33]:
        for alphabet in [1, 2, 5, 40]:
            X = rand_sorted(rng, length, dtype, alphabet)
            probes = {int(v) if dtype != np.float32 else float(v) for v in X.tolist()}
            if length:
                probes |= {X.tolist()[0] - 1, X.tolist()[-1] + 1}
            info = np.finfo(dtype) if dtype == np.float32 else np.iinfo(dtype)
            for x in sorted(probes):
                if not (info.min <= x <= info.max):
                    continue
                x = np.array(x).astype(dtype)
                lo = oracle.rank_low(x, X)
                hi = oracle.rank_high(x, X)
                assert lo == int(np.sum(X < x))
                assert hi == int(np.sum(X <= x))
                # The defining inequalities with the sentinels X[-1] = -inf, X[len] = +inf.
                assert (lo == 0 or X[lo - 1] < x) and (lo == length or x <= X[lo])
                assert (hi == 0 or X[hi - 1] <= x) and (hi == length or x < X[hi])


def test_rank_key_orders():
    # u32 compares unsigned, i32 signed, f32 by IEEE (-0.0 == +0.0).
    X = np.array([1, 5, 0x80000000, 0xFFFFFFFF], dtype=np.uint32)
    assert oracle.rank_low(np.uint32(0x90000000), X) == 3
    Xi = np.array([-7, -1, 0, 3], dtype=np.int32)
    assert oracle.rank_low(np.int32(-2), Xi) == 1
    assert oracle.rank_high(np.int32(-1), Xi) == 2
    Xf = np.array([-1.5, -0.0, 0.0, 2.0], dtype=np.float32)
    assert oracle.rank_low(np.float32(0.0), Xf) == 1
    assert oracle.rank_high(np.float32(-0.0), Xf) == 3
    Xu = np.array([1, 1 << 40, (1 << 64) - 1], dtype=np.uint64)
    assert oracle.rank_high(np.uint64((1 << 63) + 5), Xu) == 2


# ---------------------------------------------------------------------------
# Block decomposition (Section 2)
# ---------------------------------------------------------------------------

def test_block_decomposition_brute_force():
    for length in range(0, 41):
        for p in range(1, 13):
            starts = [oracle.block_start(length, p, i) for i in range(p + 1)]
            assert starts[0] == 0 and starts[p] == length
            sizes = [starts[i + 1] - starts[i] for i in range(p)]
            r = length % p
            assert sizes == [-(-length // p)] * r + [length // p] * (p - r)
            for k in range(length):
                owner = [i for i in range(p) if starts[i] <= k < starts[i + 1]]
                assert owner == [oracle.block_of(length, p, k)]
            assert oracle.block_of(length, p, length) == p


# ---------------------------------------------------------------------------
# Merges against Python's stable sort
# ---------------------------------------------------------------------------

def all_sorted_sequences(max_len, alphabet):
    for length in range(max_len + 1):
        for combo in itertools.combinations_with_replacement(range(alphabet), length):
            yield np.array(combo, dtype=np.uint32)


def test_two_pointer_exhaustive_tiny():
    seqs = list(all_sorted_sequences(4, 3))
    for A in seqs:
        for B in seqs:
            Av, Bv = payloads(len(A), len(B))
            C, Cv = oracle.merge_two_pointer(A, Av, B, Bv)
            K, V = stable_reference(A, B)
            assert np.array_equal(C, K) and np.array_equal(Cv, V)


@pytest.mark.parametrize("dtype", DTYPES)
def test_merges_random_against_stable_sort(dtype):
    rng = np.random.default_rng(5)
    for trial in range(60):
        n = int(rng.integers(0, 400))
        m = int(rng.integers(0, 400))
        alphabet = int(rng.choice([1, 3, 17, 1000]))
        A = rand_sorted(rng, n, dtype, alphabet)
        B = rand_sorted(rng, m, dtype, alphabet)
        Av, Bv = payloads(n, m)
        K, V = stable_reference(A, B)
        for fn in (oracle.merge_two_pointer, oracle.merge_rank_scatter):
            C, Cv = fn(A, Av, B, Bv)
            assert np.array_equal(C, K) and np.array_equal(Cv, V), fn.__name__


def test_merge_special_cases():
    A = np.array([3, 4, 9], dtype=np.uint32)
    B = np.array([10, 12], dtype=np.uint32)
    Av, Bv = payloads(3, 2)
    for fn in (oracle.merge_two_pointer, oracle.merge_rank_scatter):
        C, Cv = fn(A, Av, B, Bv)               # max A < min B: A || B
        assert C.tolist() == [3, 4, 9, 10, 12] and Cv.tolist() == Av.tolist() + Bv.tolist()
        C, Cv = fn(B, Bv, A, Av)               # max B < min A: B || A
        assert C.tolist() == [3, 4, 9, 10, 12] and Cv.tolist() == Av.tolist() + Bv.tolist()
        E = np.full(5, 7, dtype=np.uint32)     # all equal: A || B
        Ev, Fv = payloads(5, 5)
        C, Cv = fn(E, Ev, E, Fv)
        assert Cv.tolist() == Ev.tolist() + Fv.tolist()
        Z = np.empty(0, dtype=np.uint32)       # empty sides: copies
        C, Cv = fn(Z, Z, A, Av)
        assert C.tolist() == A.tolist()
        C, Cv = fn(A, Av, Z, Z)
        assert Cv.tolist() == Av.tolist()


def test_signed_zero_ties():
    A = np.array([-0.0, 1.0], dtype=np.float32)
    B = np.array([0.0, 0.0], dtype=np.float32)
    Av, Bv = payloads(2, 2)
    C, Cv = oracle.merge_two_pointer(A, Av, B, Bv)
    assert Cv.tolist() == [Av[0], Bv[0], Bv[1], Av[1]]   # -0.0 == 0.0: A first


# ---------------------------------------------------------------------------
# The paper's algorithm (Steps 1-4, five cases) on the host
# ---------------------------------------------------------------------------

def check_table(A, B, p, xbar, ybar, table):
    n, m = len(A), len(B)
    ca, cb, cc = np.zeros(n, int), np.zeros(m, int), np.zeros(n + m, int)
    cap = -(-n // p) + -(-m // p)
    xs = [oracle.block_start(n, p, i) for i in range(p + 1)]
    ys = [oracle.block_start(m, p, j) for j in range(p + 1)]
    for k, (lo, hi, olo, ohi, c0, case) in enumerate(table):
        assert chr(case) in "abcde"
        assert 0 <= lo <= hi and 0 <= olo <= ohi
        if k < p:
            a0, a1, b0, b1 = lo, hi, olo, ohi
            assert lo == xs[k] and olo == xbar[k]
        else:
            a0, a1, b0, b1 = olo, ohi, lo, hi
            assert lo == ys[k - p] and olo == ybar[k - p]
        assert c0 == a0 + b0                          # on the merge path
        ca[a0:a1] += 1
        cb[b0:b1] += 1
        cc[c0:c0 + (a1 - a0) + (b1 - b0)] += 1
        # each range lies inside one block (Section 2, correctness argument)
        if a1 > a0:
            assert oracle.block_of(n, p, a0) == oracle.block_of(n, p, a1 - 1)
        if b1 > b0:
            assert oracle.block_of(m, p, b0) == oracle.block_of(m, p, b1 - 1)
        assert (a1 - a0) + (b1 - b0) <= cap
        # every A element of the range precedes every B element after it, etc.
        if a1 > a0 and b0 > 0:
            assert B[b0 - 1] < A[a0]
        if b1 > b0 and a0 > 0:
            assert A[a0 - 1] <= B[b0]
    assert (ca == 1).all() and (cb == 1).all() and (cc == 1).all()


def test_paper_merge_exhaustive_small():
    rng = np.random.default_rng(3)
    for n in range(0, 13):
        for m in range(0, 13):
            for p in range(1, 13):
                for alphabet in (1, 3, 50):
                    A = rand_sorted(rng, n, np.uint32, alphabet)
                    B = rand_sorted(rng, m, np.uint32, alphabet)
                    Av, Bv = payloads(n, m)
                    C, Cv, xbar, ybar, table = oracle.paper_merge(A, Av, B, Bv, p)
                    K, V = stable_reference(A, B)
                    assert np.array_equal(C, K) and np.array_equal(Cv, V), (n, m, p)
                    check_table(A, B, p, xbar, ybar, table)


@pytest.mark.parametrize("dtype", DTYPES)
def test_paper_merge_random_larger(dtype):
    rng = np.random.default_rng(9)
    for trial in range(40):
        n = int(rng.integers(0, 3000))
        m = int(rng.integers(0, 3000))
        p = int(rng.integers(1, 200))
        alphabet = int(rng.choice([1, 4, 64, 10**6]))
        A = rand_sorted(rng, n, dtype, alphabet)
        B = rand_sorted(rng, m, dtype, alphabet)
        Av, Bv = payloads(n, m)
        C, Cv, xbar, ybar, table = oracle.paper_merge(A, Av, B, Bv, p)
        C2, Cv2 = oracle.merge_two_pointer(A, Av, B, Bv)
        assert np.array_equal(C, C2) and np.array_equal(Cv, Cv2)
        check_table(A, B, p, xbar, ybar, table)


@pytest.mark.parametrize("dtype", DTYPES)
def test_parallel_baseline_equals_oracle(dtype):
    """The CPU baseline (the paper's algorithm on POSIX threads) against the
    stable sort of the tagged concatenation and the sequential paper_merge's
    cross ranks, for thread counts below, at and above p."""
    rng = np.random.default_rng(21)
    for trial in range(30):
        n = int(rng.integers(0, 5000))
        m = int(rng.integers(0, 5000))
        p = int(rng.integers(1, 100))
        threads = int(rng.choice([1, 2, 3, 8, p, p + 5]))
        A = rand_sorted(rng, n, dtype, int(rng.choice([1, 5, 1000, 10**6])))
        B = rand_sorted(rng, m, dtype, int(rng.choice([1, 5, 1000, 10**6])))
        Av, Bv = payloads(n, m)
        C, Cv, xbar, ybar = oracle.paper_merge_parallel(A, Av, B, Bv, p, threads)
        K, V = stable_reference(A, B)
        assert np.array_equal(C, K) and np.array_equal(Cv, V), (n, m, p, threads)
        _, _, xs, ys, _ = oracle.paper_merge(A, Av, B, Bv, p)
        assert np.array_equal(xbar, xs) and np.array_equal(ybar, ys)


def test_all_equal_cross_ranks():
    # All keys equal: xbar_i = 0 (no B element is below), ybar_j = n.
    A = np.zeros(10, dtype=np.int32)
    B = np.zeros(7, dtype=np.int32)
    xbar, ybar = oracle.cross_ranks(A, B, 3)
    assert xbar.tolist() == [0, 0, 0, 7] and ybar.tolist() == [10, 10, 10, 10]


def test_observation1_cross_ranks_do_not_cross():
    rng = np.random.default_rng(1)
    for trial in range(30):
        A = rand_sorted(rng, int(rng.integers(1, 60)), np.uint32, 12)
        B = rand_sorted(rng, int(rng.integers(1, 60)), np.uint32, 12)
        for i in range(len(A)):
            j = oracle.rank_low(A[i], B)
            for jp in range(len(B)):
                hr = oracle.rank_high(B[jp], A)
                if jp < j:
                    assert hr <= i
                if jp >= j:
                    assert hr > i


# ---------------------------------------------------------------------------
# Many merges and the merge sort (Section 3)
# ---------------------------------------------------------------------------

def test_merge_batched_against_stable_sort():
    rng = np.random.default_rng(4)
    pairs = 40
    ln_a = rng.integers(0, 30, size=pairs)
    ln_b = rng.integers(0, 30, size=pairs)
    a_off = np.concatenate([[0], np.cumsum(ln_a)])
    b_off = np.concatenate([[0], np.cumsum(ln_b)])
    A = np.concatenate([rand_sorted(rng, k, np.uint64, 9) for k in ln_a])
    B = np.concatenate([rand_sorted(rng, k, np.uint64, 9) for k in ln_b])
    Av = np.arange(len(A), dtype=np.uint32)
    Bv = np.arange(len(B), dtype=np.uint32) | np.uint32(1 << 31)
    C, Cv = oracle.merge_batched(a_off, A, Av, b_off, B, Bv)
    for k in range(pairs):
        a = A[a_off[k]:a_off[k + 1]]
        b = B[b_off[k]:b_off[k + 1]]
        items = sorted([(a[i], Av[a_off[k] + i]) for i in range(len(a))]
                       + [(b[j], Bv[b_off[k] + j]) for j in range(len(b))], key=lambda t: t[0])
        c0 = a_off[k] + b_off[k]
        seg = slice(c0, c0 + len(items))
        assert C[seg].tolist() == [t[0] for t in items]
        assert Cv[seg].tolist() == [t[1] for t in items]


@pytest.mark.parametrize("run", [1, 4, 16, 1024])
@pytest.mark.parametrize("n", [0, 1, 2, 7, 100, 1000, 5000])
def test_merge_sort_against_stable_sort(run, n):
    rng = np.random.default_rng(n + run)
    keys = rng.integers(0, 50, size=n).astype(np.uint64)
    vals = np.arange(n, dtype=np.uint32)
    K, V = oracle.merge_sort(keys, vals, run)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(K, keys[order]) and np.array_equal(V, vals[order])
    ref = sorted(zip(keys.tolist(), vals.tolist()), key=lambda t: t[0])
    assert K.tolist() == [k for k, _ in ref] and V.tolist() == [v for _, v in ref]


# ---------------------------------------------------------------------------
# The property check used at sizes no reference output fits (tests/helpers)
# ---------------------------------------------------------------------------

def test_property_check_accepts_the_oracle_and_rejects_planted_mistakes():
    import torch
    from tests.helpers import stable_merge_violation
    rng = np.random.default_rng(31)
    for alphabet, dtype, unsigned in ((1 << 30, np.int32, False), (50, np.int32, False), (1, np.int32, False),
                                      (1 << 31, np.uint32, True), (1000, np.float32, False)):
        n, m = 300001, 200003
        A = rand_sorted(rng, n, dtype, alphabet)
        B = rand_sorted(rng, m, dtype, alphabet)
        Av, Bv = payloads(n, m)
        C, Cv = oracle.merge_two_pointer(A, Av, B, Bv)
        as_t = lambda x: torch.from_numpy(x.view(np.int32) if x.dtype == np.uint32 else x)
        tA, tB, tC, tCv = as_t(A), as_t(B), as_t(C), as_t(Cv)
        assert stable_merge_violation(tA, tB, tC, tCv, unsigned=unsigned, chunk=1 << 16) is None
        # an A and a B element with the same key exchanged (B before A on a tie)
        if alphabet <= 50:
            k = next(k for k in range(n + m - 1) if C[k] == C[k + 1] and (Cv[k] >> 31) == 0 and (Cv[k + 1] >> 31) == 1)
            bad = tCv.clone()
            bad[k], bad[k + 1] = tCv[k + 1], tCv[k]
            assert stable_merge_violation(tA, tB, tC, bad, unsigned=unsigned)[0] == k
        # an element duplicated in place of its neighbour (one input lost)
        bad_k, bad_v = tC.clone(), tCv.clone()
        bad_k[70000], bad_v[70000] = tC[69999], tCv[69999]
        assert stable_merge_violation(tA, tB, bad_k, bad_v, unsigned=unsigned, chunk=1 << 16)[0] == 69999
        # a payload that does not travel with its key
        bad_v = tCv.clone()
        bad_v[123457] = tCv[123457] ^ 1 if (int(tCv[123457]) & 0x7FFFFFFF) ^ 1 < n else tCv[123457] - 1
        assert stable_merge_violation(tA, tB, tC, bad_v, unsigned=unsigned) is not None
        # a key one unit off at a chunk boundary
        if dtype != np.float32:
            bad_k = tC.clone()
            bad_k[1 << 16] += 1
            assert stable_merge_violation(tA, tB, bad_k, tCv, unsigned=unsigned, chunk=1 << 16)[0] == 1 << 16


def test_sort_property_check_accepts_the_oracle_and_rejects_planted_mistakes():
    import torch
    from tests.helpers import stable_sort_violation
    rng = np.random.default_rng(33)
    n = 400003
    for keys, unsigned in ((rng.integers(0, 1 << 24, size=n).astype(np.uint64), False),
                           (rng.integers(0, 7, size=n).astype(np.uint64), False),
                           (rng.integers(0, 1 << 32, size=n).astype(np.uint32), True)):
        vals = np.arange(n, dtype=np.uint32)
        K, V = oracle.merge_sort(keys, vals, run=16)
        assert np.array_equal(K, keys[np.argsort(keys, kind="stable")])
        as_t = lambda x: torch.from_numpy(x.view(np.int64) if x.dtype == np.uint64 else x.view(np.int32))
        tS, tK, tV = as_t(keys), as_t(K), as_t(V)
        assert stable_sort_violation(tS, tK, tV, unsigned=unsigned, chunk=1 << 16) is None
        eq = np.nonzero(K[1:] == K[:-1])[0]
        k = int(eq[len(eq) // 2])                       # two equal keys out of input order
        bad = tV.clone()
        bad[k], bad[k + 1] = tV[k + 1], tV[k]
        assert stable_sort_violation(tS, tK, bad, unsigned=unsigned, chunk=1 << 16)[0] == k
        bad = tV.clone()                                 # an index used twice, another lost
        bad[(1 << 16) + 5] = tV[(1 << 16) + 4]
        assert stable_sort_violation(tS, tK, bad, unsigned=unsigned, chunk=1 << 16) is not None
        bad = tK.clone()                                 # keys out of order at a chunk boundary
        bad[1 << 16], bad[(1 << 16) - 1] = tK[(1 << 16) - 1], tK[1 << 16]
        if K[1 << 16] != K[(1 << 16) - 1]:
            assert stable_sort_violation(tS, bad, tV, unsigned=unsigned, chunk=1 << 16) is not None
