"""The library's block arithmetic of Section 2 (block starts, block of an
index, first block starting at or after an index, and the division with its
32-bit fast path), compiled for the host from the same header the kernels
use, against the oracle and exact integer arithmetic: exhaustively on small
sizes and at sizes up to 2^62 that no GPU test can allocate.  No GPU is
used (nvcc cross-compiles the harness; only host code runs).
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HARNESS = os.path.join(ROOT, "tests", "host", "block_arith.cu")


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cc = _nvcc()
    if cc is None:
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("host_arith") / "libblock_arith.so")
    subprocess.check_call([cc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                           "-Xcompiler", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_1202_6575_gb300", "csrc"),
                           HARNESS, "-o", out])
    L = ctypes.CDLL(out)
    i64, i32 = ctypes.c_int64, ctypes.c_int32
    for name, t in (("h_div_nonneg64", i64), ("h_block_start64", i64), ("h_block_of64", i64),
                    ("h_first_block64", i64)):
        f = getattr(L, name)
        f.restype = t
        f.argtypes = [t] * (2 if "div" in name else 3)
    for name in ("h_div_nonneg32", "h_block_start32"):
        f = getattr(L, name)
        f.restype = i32
        f.argtypes = [i32] * (2 if "div" in name else 3)
    u32 = ctypes.c_uint32
    L.h_fastdiv32.restype = u32
    L.h_fastdiv32.argtypes = [u32, u32]
    for name in ("h_blocks32_start", "h_blocks32_of", "h_blocks32_first"):
        f = getattr(L, name)
        f.restype = i64
        f.argtypes = [u32, u32, i64]
    return L


def first_block_brute(length, p, k):
    """Smallest j with block start y_j >= k, by bisection over the oracle's
    (non-decreasing) block starts; for k = len with len < p the first empty
    block, j = len (its start is len)."""
    lo, hi = 0, p
    while lo < hi:
        mid = (lo + hi) // 2
        if oracle.block_start(length, p, mid) >= k:
            hi = mid
        else:
            lo = mid + 1
    return lo


def test_small_sizes_exhaustive_against_the_oracle(lib):
    for length in range(0, 41):
        for p in range(1, 14):
            for i in range(p + 1):
                assert lib.h_block_start64(length, p, i) == oracle.block_start(length, p, i)
                assert lib.h_block_start32(length, p, i) == oracle.block_start(length, p, i)
            for k in range(length + 1):
                assert lib.h_block_of64(length, p, k) == oracle.block_of(length, p, k), (length, p, k)
                assert lib.h_first_block64(length, p, k) == first_block_brute(length, p, k), (length, p, k)


def test_large_sizes_against_exact_integers(lib):
    rng = np.random.default_rng(11)
    cases = []
    for e_len in (31, 32, 33, 40, 50, 62):
        for _ in range(60):
            length = int(rng.integers(1 << (e_len - 1), (1 << e_len) + 1))
            p = int(rng.choice([1, 2, 3, 1023, 1024, 65537, (1 << 31) - 1, 1 << 31, (1 << 32) + 3]))
            p = max(1, min(p, length + 5))
            cases.append((length, p))
    cases += [((1 << 62) - 1, (1 << 31) - 1), ((1 << 32) - 1, 1 << 16), (1 << 32, 1 << 16),
              ((1 << 32) + 1, 3), (5, 1 << 40)]
    for length, p in cases:
        q, r = divmod(length, p)
        for i in sorted(i for i in {0, 1, r - 1, r, r + 1, p // 2, p - 1, p} if 0 <= i <= p):
            exact = i * (q + 1) if i < r else i * q + r       # first r blocks hold q + 1 elements
            assert lib.h_block_start64(length, p, i) == exact, (length, p, i)
            if i < p and exact < length:
                assert lib.h_block_of64(length, p, exact) == i
                nxt = i * (q + 1) + q + 1 if i < r else (i + 1) * q + r
                assert lib.h_block_of64(length, p, nxt - 1) == i
                assert lib.h_first_block64(length, p, exact) == i
                if nxt - exact > 1:
                    assert lib.h_first_block64(length, p, exact + 1) == i + 1
        assert lib.h_block_of64(length, p, length) == p
        assert lib.h_first_block64(length, p, length) == (length if length < p else p)


def test_division_fast_path_boundaries(lib):
    vals = [0, 1, 2, 3, 7, (1 << 31) - 1, 1 << 31, (1 << 32) - 2, (1 << 32) - 1, 1 << 32, (1 << 32) + 1,
            (1 << 40) + 12345, (1 << 62) - 1, (1 << 63) - 1]
    for a in vals:
        for b in vals[1:]:
            assert lib.h_div_nonneg64(a, b) == a // b, (a, b)
    for a in (0, 1, 5, (1 << 31) - 1):
        for b in (1, 2, 3, (1 << 31) - 1):
            assert lib.h_div_nonneg32(a, b) == a // b


def test_invariant_divisor_division_against_exact_integers(lib):
    """FastDiv32 (division by an invariant divisor through a 64-bit
    reciprocal, Lemire, Kaser and Kurz 2019) equals floor(x / d) for 32-bit
    x and d: every divisor up to 300 against every x up to 2000, and random
    and boundary pairs over the whole range."""
    for d in range(1, 301):
        for x in list(range(0, 2001)) + [(1 << 32) - 1, (1 << 32) - d, (1 << 31) + 7]:
            assert lib.h_fastdiv32(x, d) == x // d, (x, d)
    rng = np.random.default_rng(5)
    edge = [1, 2, 3, 5, 7, 641, 65535, 65536, 65537, (1 << 31) - 1, 1 << 31, (1 << 31) + 1, (1 << 32) - 1]
    xs = [int(v) for v in rng.integers(0, 1 << 32, 4000)] + [0, 1, (1 << 32) - 1, (1 << 31), (1 << 31) - 1]
    ds = [int(v) for v in rng.integers(1, 1 << 32, 400)] + edge + [1 << k for k in range(32)]
    for d in ds:
        for x in xs[:200] + [d - 1, d, d + 1, 2 * d - 1, 2 * d] if d < (1 << 31) else xs[:200]:
            if x < (1 << 32):
                assert lib.h_fastdiv32(x, d) == x // d, (x, d)
    for x in xs:
        d = int(rng.choice(ds))
        assert lib.h_fastdiv32(x, d) == x // d, (x, d)


def test_blocks32_equals_the_general_block_arithmetic(lib):
    """The fused launch's precomputed 32-bit block decomposition (Blocks32)
    against the oracle exhaustively on small sizes and against the general
    64-bit functions on random sizes below 2^31."""
    for length in range(0, 41):
        for p in range(1, 14):
            for i in range(p + 1):
                assert lib.h_blocks32_start(length, p, i) == oracle.block_start(length, p, i)
            for k in range(length + 1):
                assert lib.h_blocks32_of(length, p, k) == oracle.block_of(length, p, k), (length, p, k)
                assert lib.h_blocks32_first(length, p, k) == first_block_brute(length, p, k), (length, p, k)
    rng = np.random.default_rng(12)
    for _ in range(300):
        length = int(rng.integers(1, 1 << 31))
        p = int(rng.choice([1, 2, 3, 1024, 16384, int(rng.integers(1, 1 << 20))]))
        ks = [0, length, length - 1] + [int(v) for v in rng.integers(0, length + 1, 20)]
        for i in [0, 1, p - 1, p] + [int(v) for v in rng.integers(0, p + 1, 10)]:
            assert lib.h_blocks32_start(length, p, i) == lib.h_block_start64(length, p, i), (length, p, i)
        for k in ks:
            assert lib.h_blocks32_of(length, p, k) == lib.h_block_of64(length, p, k), (length, p, k)
            assert lib.h_blocks32_first(length, p, k) == lib.h_first_block64(length, p, k), (length, p, k)


def _selection(lib, width, n, m, p, xbar, ybar):
    f = lib.h_all_subproblems32 if width == 32 else lib.h_all_subproblems64
    t = ctypes.c_int32 if width == 32 else ctypes.c_int64
    P = ctypes.c_void_p
    f.restype = None
    f.argtypes = [t, t, t, P, P, P]
    out = np.zeros((2 * p, 5), dtype=np.int64)
    xb, yb = np.ascontiguousarray(xbar, dtype=np.int64), np.ascontiguousarray(ybar, dtype=np.int64)
    f(n, m, p, xb.ctypes.data, yb.ctypes.data, out.ctypes.data)
    return out


def _closed_form_ranks(n, m, p, c1, d1, c2, d2):
    """Cross ranks of A[i] = floor(i c1 / d1) (n keys) and B[j] = floor(j c2 /
    d2) (m keys), exactly, without the arrays: #{j : B[j] < v} = min(m,
    ceil(v d2 / c2)) and #{i : A[i] <= v} = min(n, ceil((v + 1) d1 / c1))."""
    xs = [oracle.block_start(n, p, k) for k in range(p)]
    ys = [oracle.block_start(m, p, k) for k in range(p)]
    xbar = [min(m, -(-((x * c1 // d1) * d2) // c2)) for x in xs] + [m]
    ybar = [min(n, -(-(((y * c2 // d2) + 1) * d1) // c1)) for y in ys] + [n]
    return np.array(xbar, dtype=np.int64), np.array(ybar, dtype=np.int64)


@pytest.mark.parametrize("n,m,p,c1,d1,c2,d2", [
    ((1 << 30) - 1, (1 << 30) - 3, 1 << 17, 3, 1, 3, 1),
    ((1 << 30) - 1, 5, 1 << 16, 1, 1, 7, 2),
    (999_999_937, 123_456_791, 40_001, 5, 3, 2, 7),
    (1 << 27, 1 << 27, 131072, 1, 16, 1, 16),
    (4097, (1 << 29) + 11, 3, 11, 2, 1, 5)])
def test_selection_in_32_bits_equals_64_bits(lib, n, m, p, c1, d1, c2, d2):
    """The batched plan kernel selects the subproblems of pairs below 2^30
    (every pair of a sort round) with 32-bit block arithmetic: the same
    records and chain indices as the 64-bit path, on exact cross ranks of
    tie-heavy and tie-free key sequences up to just below 2^30."""
    xbar, ybar = _closed_form_ranks(n, m, p, c1, d1, c2, d2)
    a = _selection(lib, 32, n, m, p, xbar, ybar)
    b = _selection(lib, 64, n, m, p, xbar, ybar)
    assert np.array_equal(a, b)


def test_selection_matches_the_oracles_five_cases_small(lib):
    """On small sizes both widths give the oracle's subproblems (its
    literal five cases) from the oracle's cross ranks."""
    rng = np.random.default_rng(3)
    for _ in range(60):
        n, m = int(rng.integers(0, 300)), int(rng.integers(0, 300))
        p = int(rng.integers(1, 40))
        A = np.sort(rng.integers(0, 20, n)).astype(np.int32)
        B = np.sort(rng.integers(0, 20, m)).astype(np.int32)
        xbar, ybar = oracle.cross_ranks(A, B, p)
        t = oracle.subproblems(n, m, p, xbar, ybar)      # rows: own range, other side's range
        want = np.concatenate([t[:p, [0, 1, 2, 3]], t[p:, [2, 3, 0, 1]]])   # as (a0, a1, b0, b1)
        for width in (32, 64):
            got = _selection(lib, width, n, m, p, xbar, ybar)
            assert np.array_equal(got[:, :4], want), (n, m, p, width)
