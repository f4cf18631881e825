"""Reference oracle for the stable parallel merge (Traeff, arXiv:1202.6575).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares
no code with the GPU library (``paper_1202_6575_gb300``) and never imports it;
the library never imports this package.

Three parts:

* ``tm_oracle.c`` (plain C, single thread, loaded through ctypes): the rank
  primitives and block decomposition of Section 2, Steps 1-4 with the five
  cases (a)-(e), the textbook stable two-pointer merge, the rank-scatter merge
  built from the position formulas of Section 2, many independent merges, and
  the stable merge sort of Section 3.
* ``paper_parallel.c`` (POSIX threads): a CPU baseline, not a reference: the
  paper's algorithm with one thread per processing element, on the oracle's
  searches, five cases and two-pointer merge (checked against them by the
  tests; the benchmark times it beside the single-thread merge).
* ``cdf.py`` (numpy, float64): the learned cross-rank model (piecewise-linear
  CDF plus a two-layer MLP) forward, loss, backward and Adam step.  This model
  is not in the paper; it proposes cross ranks that the exact search then
  verifies.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tm_oracle.c")
_SRC_PAR = os.path.join(_HERE, "paper_parallel.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
# A prebuilt copy of the oracle library to load instead of building this one:
# tests/test_oracle_mutants.py points it at copies with one planted mistake
# each, to show that the pins catch every such mistake.
_LIB_OVERRIDE = os.environ.get("TM_ORACLE_LIB")

_KEY_SUFFIX = {
    np.dtype(np.uint32): "u32",
    np.dtype(np.int32): "i32",
    np.dtype(np.uint64): "u64",
    np.dtype(np.float32): "f32",
}
_KEY_CTYPE = {
    "u32": ctypes.c_uint32,
    "i32": ctypes.c_int32,
    "u64": ctypes.c_uint64,
    "f32": ctypes.c_float,
}

_lib = None


def build(force: bool = False) -> str:
    """Compile tm_oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_PAR))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-pthread",
                           "-o", tmp, _SRC, _SRC_PAR])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        if _LIB_OVERRIDE:
            _lib = ctypes.CDLL(_LIB_OVERRIDE)
        else:
            build()
            _lib = ctypes.CDLL(_LIB_PATH)
        i64, p = ctypes.c_int64, ctypes.c_void_p
        _lib.orc_block_start.restype = i64
        _lib.orc_block_start.argtypes = [i64, i64, i64]
        _lib.orc_block_of.restype = i64
        _lib.orc_block_of.argtypes = [i64, i64, i64]
        _lib.orc_subproblems.restype = None
        _lib.orc_subproblems.argtypes = [i64, i64, i64, p, p, p]
        for s, ct in _KEY_CTYPE.items():
            for name in ("rank_low", "rank_high"):
                f = getattr(_lib, f"orc_{name}_{s}")
                f.restype = i64
                f.argtypes = [ct, p, i64]
            for name in ("merge_two_pointer", "merge_rank_scatter"):
                f = getattr(_lib, f"orc_{name}_{s}")
                f.restype = None
                f.argtypes = [p, p, i64, p, p, i64, p, p]
            f = getattr(_lib, f"orc_cross_ranks_{s}")
            f.restype = None
            f.argtypes = [p, i64, p, i64, i64, p, p]
            f = getattr(_lib, f"orc_paper_merge_{s}")
            f.restype = None
            f.argtypes = [p, p, i64, p, p, i64, i64, p, p, p, p, p]
            f = getattr(_lib, f"orc_paper_merge_parallel_{s}")
            f.restype = ctypes.c_int
            f.argtypes = [p, p, i64, p, p, i64, i64, i64, p, p, p, p]
            f = getattr(_lib, f"orc_merge_batched_{s}")
            f.restype = None
            f.argtypes = [i64, p, p, p, p, p, p, p, p]
            f = getattr(_lib, f"orc_merge_sort_{s}")
            f.restype = None
            f.argtypes = [p, p, i64, i64, p, p]
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _suffix(keys: np.ndarray) -> str:
    try:
        return _KEY_SUFFIX[keys.dtype]
    except KeyError:
        raise TypeError(f"unsupported key dtype {keys.dtype}") from None


def _c(a: np.ndarray, dtype=None) -> np.ndarray:
    return np.ascontiguousarray(a if dtype is None else a.astype(dtype, copy=False))


# --------------------------------------------------------------------------
# Section 2: block decomposition and rank primitives
# --------------------------------------------------------------------------

def block_start(length: int, p: int, i: int) -> int:
    """x_i of the block decomposition (Section 2); x_p = length."""
    return int(_load().orc_block_start(length, p, i))


def block_of(length: int, p: int, k: int) -> int:
    """Block holding index k by the O(1) rule of Section 2; k = length -> p."""
    return int(_load().orc_block_of(length, p, k))


def rank_low(x, X: np.ndarray) -> int:
    """rank_low(x, X): the i with X[i-1] < x <= X[i] (Section 2)."""
    X = _c(X)
    s = _suffix(X)
    return int(getattr(_load(), f"orc_rank_low_{s}")(_KEY_CTYPE[s](x), _ptr(X), len(X)))


def rank_high(x, X: np.ndarray) -> int:
    """rank_high(x, X): the j with X[j-1] <= x < X[j] (Section 2)."""
    X = _c(X)
    s = _suffix(X)
    return int(getattr(_load(), f"orc_rank_high_{s}")(_KEY_CTYPE[s](x), _ptr(X), len(X)))


# --------------------------------------------------------------------------
# Merges
# --------------------------------------------------------------------------

def _merge_call(name, A, Av, B, Bv):
    A, B = _c(A), _c(B)
    if A.dtype != B.dtype:
        raise TypeError("A and B keys must have one dtype")
    Av, Bv = _c(Av, np.uint32), _c(Bv, np.uint32)
    n, m = len(A), len(B)
    C = np.empty(n + m, dtype=A.dtype)
    Cv = np.empty(n + m, dtype=np.uint32)
    getattr(_load(), f"orc_{name}_{_suffix(A)}")(
        _ptr(A), _ptr(Av), n, _ptr(B), _ptr(Bv), m, _ptr(C), _ptr(Cv))
    return C, Cv


def merge_two_pointer(A, Av, B, Bv):
    """Textbook stable merge; equal keys: A first."""
    return _merge_call("merge_two_pointer", A, Av, B, Bv)


def merge_rank_scatter(A, Av, B, Bv):
    """Merge by the position formulas of Section 2 (i + rank_low(A[i], B),
    j + rank_high(B[j], A))."""
    return _merge_call("merge_rank_scatter", A, Av, B, Bv)


def cross_ranks(A, B, p: int):
    """Steps 1 and 2: (xbar[0..p], ybar[0..p])."""
    A, B = _c(A), _c(B)
    xbar = np.empty(p + 1, dtype=np.int64)
    ybar = np.empty(p + 1, dtype=np.int64)
    getattr(_load(), f"orc_cross_ranks_{_suffix(A)}")(
        _ptr(A), len(A), _ptr(B), len(B), p, _ptr(xbar), _ptr(ybar))
    return xbar, ybar


def subproblems(n: int, m: int, p: int, xbar, ybar) -> np.ndarray:
    """Steps 3 and 4 (five cases).  Returns int64[2p, 6] rows
    (lo, hi, other_lo, other_hi, c_lo, case) -- rows < p are A-side (own
    range in A, other in B), rows >= p are B-side (own in B, other in A)."""
    xbar = _c(xbar, np.int64)
    ybar = _c(ybar, np.int64)
    table = np.empty((2 * p, 6), dtype=np.int64)
    _load().orc_subproblems(n, m, p, _ptr(xbar), _ptr(ybar), _ptr(table))
    return table


def paper_merge(A, Av, B, Bv, p: int):
    """The paper's algorithm on the host: Steps 1-4, each subproblem merged
    by the two-pointer merge.  Returns (C, Cv, xbar, ybar, table)."""
    A, B = _c(A), _c(B)
    Av, Bv = _c(Av, np.uint32), _c(Bv, np.uint32)
    n, m = len(A), len(B)
    C = np.empty(n + m, dtype=A.dtype)
    Cv = np.empty(n + m, dtype=np.uint32)
    xbar = np.empty(p + 1, dtype=np.int64)
    ybar = np.empty(p + 1, dtype=np.int64)
    table = np.empty((2 * p, 6), dtype=np.int64)
    getattr(_load(), f"orc_paper_merge_{_suffix(A)}")(
        _ptr(A), _ptr(Av), n, _ptr(B), _ptr(Bv), m, p,
        _ptr(C), _ptr(Cv), _ptr(xbar), _ptr(ybar), _ptr(table))
    return C, Cv, xbar, ybar, table


def paper_merge_parallel(A, Av, B, Bv, p: int, threads: int):
    """CPU baseline (paper_parallel.c): the paper's algorithm with one POSIX
    thread per processing element (threads of them, PE t also taking
    t + threads, ...): Steps 1-2, the synchronisation, Steps 3-4 and the
    subproblem merges.  Returns (C, Cv, xbar, ybar)."""
    A, B = _c(A), _c(B)
    Av, Bv = _c(Av, np.uint32), _c(Bv, np.uint32)
    n, m = len(A), len(B)
    C = np.empty(n + m, dtype=A.dtype)
    Cv = np.empty(n + m, dtype=np.uint32)
    xbar = np.empty(p + 1, dtype=np.int64)
    ybar = np.empty(p + 1, dtype=np.int64)
    rc = getattr(_load(), f"orc_paper_merge_parallel_{_suffix(A)}")(
        _ptr(A), _ptr(Av), n, _ptr(B), _ptr(Bv), m, p, threads,
        _ptr(C), _ptr(Cv), _ptr(xbar), _ptr(ybar))
    if rc != 0:
        raise MemoryError("paper_merge_parallel: no memory for its thread table")
    return C, Cv, xbar, ybar


def merge_batched(a_off, A, Av, b_off, B, Bv):
    """Independent stable merges of CSR pairs; pair k's output starts at
    a_off[k] + b_off[k]."""
    a_off = _c(a_off, np.int64)
    b_off = _c(b_off, np.int64)
    A, B = _c(A), _c(B)
    Av, Bv = _c(Av, np.uint32), _c(Bv, np.uint32)
    pairs = len(a_off) - 1
    C = np.empty(len(A) + len(B), dtype=A.dtype)
    Cv = np.empty(len(A) + len(B), dtype=np.uint32)
    getattr(_load(), f"orc_merge_batched_{_suffix(A)}")(
        pairs, _ptr(a_off), _ptr(A), _ptr(Av), _ptr(b_off), _ptr(B), _ptr(Bv),
        _ptr(C), _ptr(Cv))
    return C, Cv


def merge_sort(keys, vals, run: int = 1):
    """Stable merge sort of Section 3 (blocks of `run` sorted sequentially,
    then pairwise merge rounds).  Returns sorted copies."""
    k = np.array(keys, copy=True)
    v = np.array(vals, dtype=np.uint32, copy=True)
    tk = np.empty_like(k)
    tv = np.empty_like(v)
    getattr(_load(), f"orc_merge_sort_{_suffix(k)}")(
        _ptr(k), _ptr(v), len(k), run, _ptr(tk), _ptr(tv))
    return k, v


# The same for the learned-model oracle: a planted copy of cdf.py replaces
# the real one as ``oracle.cdf`` when TM_ORACLE_CDF names it.
_CDF_OVERRIDE = os.environ.get("TM_ORACLE_CDF")
if _CDF_OVERRIDE:
    import importlib.util
    import sys

    _spec = importlib.util.spec_from_file_location(__name__ + ".cdf", _CDF_OVERRIDE)
    cdf = importlib.util.module_from_spec(_spec)
    sys.modules[_spec.name] = cdf
    _spec.loader.exec_module(cdf)
