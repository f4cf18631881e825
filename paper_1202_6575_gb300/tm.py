"""Python binding of libtm.so, the C ABI declared in include/tm.h.

Argument marshalling only: every function here checks tensor devices, dtypes
and contiguity, turns tensors into device pointers and the current torch
stream into a cudaStream_t, and calls the C entry point of the same name.
All computation runs in the library's CUDA kernels.  There is no CPU path:
if libtm.so is missing or no CUDA device is present, calls raise.

A call given `stream` allocates (and zero-fills) the tensors it makes itself
-- outputs, temporaries, workspaces -- on that stream, so that the caching
allocator orders their reuse after the call's kernels.  Inputs are the
caller's: work on another stream that produced them must be ordered before
the call (stream.wait_stream), as for any torch operation.
"""
from __future__ import annotations

import ctypes
import functools
import inspect
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtm.so")

KEY_TYPES = {"u32": 0, "i32": 1, "u64": 2, "f32": 3}
KEY_BYTES = {"u32": 4, "i32": 4, "u64": 8, "f32": 4}
TORCH_KEY_DTYPES = {"u32": (torch.int32,), "i32": (torch.int32,), "u64": (torch.int64,),
                    "f32": (torch.float32,)}

TM_OK = 0
TM_ERR_INVALID = 1
TM_ERR_UNSUPPORTED = 2
TM_ERR_WORKSPACE = 3
TM_ERR_CUDA = 4
TM_ERR_TIMEOUT = 5
TM_ERR_BOUNDS = 6
TM_PARTITION_BLOCKS = 0
TM_PARTITION_DIAGONALS = 1

SPLIT_BLOCKS = 1
SPLIT_DIAGONAL = 2

# Payloads are opaque 32-bit words (int32 tensors; uint32 where torch has it).
PAYLOAD_DTYPES = (torch.int32,) + ((torch.uint32,) if hasattr(torch, "uint32") else ())


class TmConfig(ctypes.Structure):
    """struct tm_config of include/tm.h (0 = default in every field)."""
    _fields_ = [("p", ctypes.c_int64), ("tile", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("stages", ctypes.c_int32), ("split", ctypes.c_int32),
                ("wait_ms", ctypes.c_int32), ("test_drop_tile", ctypes.c_int32), ("unfused", ctypes.c_int32),
                ("partition", ctypes.c_int32), ("payload_bytes", ctypes.c_int32), ("trace", ctypes.c_int32),
                ("merge_ways", ctypes.c_int32)]


class TmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {tm_status_str(code)} (status {code})")


_lib = None
_I64, _I32, _SZ, _P = ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t, ctypes.c_void_p

# name -> (restype, argtypes); the ABI of include/tm.h.
_SIGNATURES = {
    "tm_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "tm_version": (ctypes.c_int, []),
    "tm_last_cuda_error": (ctypes.c_char_p, []),
    "tm_read_status": (ctypes.c_int, [_P, _P]),
    "tm_merge_blocks": (_I64, [_I64, _I64, _P]),
    "tm_merge_workspace_size": (_SZ, [_I64, _I64, _P]),
    "tm_merge": (ctypes.c_int, [ctypes.c_int, _P, _P, _I64, _P, _P, _I64, _P, _P, _P, _SZ, _P, _P]),
    "tm_cross_ranks": (ctypes.c_int, [ctypes.c_int, _P, _I64, _P, _I64, _I64, _P, _P, _P]),
    "tm_tile_record_bytes": (_SZ, []),
    "tm_merge_tile_cap": (_I32, [_I64, _I64, _I64]),
    "tm_plan_tile_count": (_I64, [_I64, _I64, _I64]),
    "tm_plan_subproblems": (ctypes.c_int, [_I64, _I64, _I64, _P, _P, _P, _P, _P]),
    "tm_merge_tiles": (ctypes.c_int, [ctypes.c_int, _P, _P, _I64, _P, _P, _I64, _P, _I64, _I32, _P, _P, _P,
                                      _P, _P]),
    "tm_rank_search": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _I64, _P, _I64, _P, _P]),
    "tm_subproblems": (ctypes.c_int, [_I64, _I64, _I64, _P, _P, _P, _P]),
    "tm_merge_noalloc": (ctypes.c_int, [ctypes.c_int, _P, _P, _I64, _P, _P, _I64, _P, _P, _P, _P, _P]),
    "tm_merge_phase_times": (ctypes.c_int, [_P, _I64, _I64, _P, _P, _P]),
    "tm_merge_trace": (ctypes.c_int, [_P, _I64, _I64, _P, _P, _I64, _P, _P]),
    "tm_merge_sort_segmented_workspace_size": (_SZ, [_I64, _P, _I64, _P]),
    "tm_merge_sort_segmented": (ctypes.c_int, [ctypes.c_int, _P, _P, _I64, _P, _I64, _P, _P, _P, _SZ, _P, _P]),
    "tm_merge_batched_workspace_size": (_SZ, [_I64, _I64, _I64, _P]),
    "tm_merge_batched": (ctypes.c_int, [ctypes.c_int, _I64, _P, _P, _P, _I64, _P, _P, _P, _I64, _P, _P, _P, _SZ,
                                        _P, _P]),
    "tm_merge_sort_workspace_size": (_SZ, [_I64, _P]),
    "tm_merge_sort": (ctypes.c_int, [ctypes.c_int, _P, _P, _I64, _P, _P, _P, _SZ, _P, _P]),
    "tm_autotune_batched": (ctypes.c_int, [ctypes.c_int, _I64, _P, _P, _P, _I64, _P, _P, _P, _I64, _P, _P, _P,
                                           _SZ, _P, _P]),
    "tm_autotune_sort": (ctypes.c_int, [ctypes.c_int, _P, _P, _I64, _P, _P, _P, _P, _P, _SZ, _P, _P]),
    "tm_autotune_clear": (ctypes.c_int, []),
    "tm_graph_capture_begin": (ctypes.c_int, [_P]),
    "tm_graph_capture_end": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_void_p)]),
    "tm_graph_launch": (ctypes.c_int, [_P, _P]),
    "tm_graph_destroy": (None, [_P]),
    "tm_cdf_model_bytes": (_SZ, [ctypes.c_int, ctypes.c_int]),
    "tm_cdf_init": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _I64, _P, _P]),
    "tm_cdf_grad": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, _I64, _P, _P, _P]),
    "tm_cdf_train": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, _I64, ctypes.c_int, ctypes.c_float,
                                    _P]),
    "tm_cdf_predict": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _I64, _P, _P]),
    "tm_cdf_calibrate": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, _I64, _P]),
    "tm_cross_ranks_learned": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _I64, _P, _I64, _I64, _P, _P,
                                              ctypes.c_int, _P]),
    "tm_merge_learned": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, _I64, _P, _P, _I64, _P, _P, _P,
                                        _SZ, _P, ctypes.c_int, _P]),
}


def load():
    """Loads libtm.so (built by paper_1202_6575_gb300.build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -m paper_1202_6575_gb300.build)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGNATURES)


def tm_status_str(code: int) -> str:
    return load().tm_status_str(int(code)).decode()


def tm_version() -> int:
    return int(load().tm_version())


def tm_last_cuda_error() -> str:
    return load().tm_last_cuda_error().decode()


def _check(code: int, where: str):
    if code != TM_OK:
        raise TmError(code, where + (f" [{tm_last_cuda_error()}]" if code == TM_ERR_CUDA else ""))


def _cfg_struct(cfg) -> TmConfig:
    """A TmConfig holding cfg (None: all defaults)."""
    c = TmConfig()
    if isinstance(cfg, TmConfig):
        ctypes.memmove(ctypes.addressof(c), ctypes.addressof(cfg), ctypes.sizeof(TmConfig))
    elif cfg:
        for k, v in dict(cfg).items():
            setattr(c, k, int(v))
    return c


def _cfg(cfg):
    if cfg is None:
        return None
    if isinstance(cfg, TmConfig):
        return ctypes.byref(cfg)
    c = TmConfig()
    for k, v in dict(cfg).items():
        setattr(c, k, int(v))
    return ctypes.byref(c)



def _on_stream(fn):
    """Runs the binding with `stream` (keyword or positional) as the current
    torch stream, so that what it allocates belongs to that stream."""
    params = list(inspect.signature(fn).parameters)
    pos = params.index("stream")

    @functools.wraps(fn)
    def wrapped(*a, **k):
        s = k.get("stream", a[pos] if len(a) > pos else None)
        if s is None:
            return fn(*a, **k)
        with torch.cuda.stream(s):
            return fn(*a, **k)
    return wrapped

def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev(t, name: str, dtypes=None) -> int:
    if t is None:                       # optional array (payloads of a keys-only call)
        return 0
    if dtypes is not None and t.dtype not in dtypes:
        raise ValueError(f"{name} has dtype {t.dtype}, expected one of {dtypes}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    return t.data_ptr() if t.numel() else 0


PAYLOAD64_DTYPES = (torch.int64,) + ((torch.uint64,) if hasattr(torch, "uint64") else ())
ANY_PAYLOAD_DTYPES = PAYLOAD_DTYPES + PAYLOAD64_DTYPES


def _payload_cfg(cfg, *vals):
    """cfg with payload_bytes set from the payload tensors' word size (8 for
    64-bit payload dtypes, else 4 as given); the tensors must agree."""
    widths = {8 if v.dtype in PAYLOAD64_DTYPES else 4 for v in vals if v is not None}
    if len(widths) > 1:
        raise ValueError("payload tensors mix 32-bit and 64-bit words")
    width = max(widths) if widths else 4
    if isinstance(cfg, TmConfig):
        given = cfg.payload_bytes                  # 0: follow the tensors
        if widths and given and given != width:
            raise ValueError(f"cfg.payload_bytes = {given} but the payloads are {width}-byte words")
        if width == 8 and given != 8:
            c = TmConfig.from_buffer_copy(cfg)
            c.payload_bytes = 8
            return c
        return cfg
    d = dict(cfg or {})
    given = d.get("payload_bytes", 0)
    if any(v is not None for v in vals) and given and given != width:
        raise ValueError(f"payload_bytes = {given} but the payloads are {width}-byte words")
    if width == 8:
        d["payload_bytes"] = 8
    return d or cfg


def _kt(kt: str) -> int:
    try:
        return KEY_TYPES[kt]
    except KeyError:
        raise ValueError(f"unknown key type {kt!r}") from None


# ---------------------------------------------------------------------------
# Single merge
# ---------------------------------------------------------------------------

def tm_merge_blocks(n: int, m: int, cfg=None) -> int:
    return int(load().tm_merge_blocks(n, m, _cfg(cfg)))


def tm_merge_workspace_size(n: int, m: int, cfg=None) -> int:
    return int(load().tm_merge_workspace_size(n, m, _cfg(cfg)))


def new_workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


@_on_stream
def tm_merge(kt: str, A, Av, B, Bv, C=None, Cv=None, workspace=None, cfg=None, stream=None):
    """Stable merge of (A, Av) and (B, Bv); returns (C, Cv, workspace).
    Av = Bv = None merges keys only (Cv None).  The status word is the first
    4 bytes of the workspace (tm_read_status)."""
    kd = TORCH_KEY_DTYPES[kt]
    n, m = A.numel(), B.numel()
    if C is None:
        C = torch.empty(n + m, dtype=A.dtype, device=A.device)
    keys_only = Av is None and Bv is None
    if Cv is None and not keys_only:
        Cv = torch.empty(n + m, dtype=(Av if Av is not None else Bv).dtype, device=A.device)
    if C.numel() != n + m or (not keys_only and (Cv.numel() != n + m or Av.numel() != n or Bv.numel() != m)):
        raise ValueError("length mismatch")
    cfg = _payload_cfg(cfg, Av, Bv, Cv)
    cfgp = _cfg(cfg)
    if workspace is None:
        workspace = new_workspace(tm_merge_workspace_size(n, m, cfg), A.device)
    code = load().tm_merge(_kt(kt), _dev(A, "A", kd), _dev(Av, "Av", ANY_PAYLOAD_DTYPES), n, _dev(B, "B", kd),
                           _dev(Bv, "Bv", ANY_PAYLOAD_DTYPES), m, _dev(C, "C", kd), _dev(Cv, "Cv", ANY_PAYLOAD_DTYPES),
                           _dev(workspace, "workspace"), workspace.numel(), cfgp, _stream(stream))
    _check(code, "tm_merge")
    return C, Cv, workspace


@_on_stream
def tm_cross_ranks(kt: str, A, B, p: int, xbar=None, ybar=None, stream=None):
    """Steps 1-2: returns (xbar, ybar), int64 tensors of p + 1 entries."""
    kd = TORCH_KEY_DTYPES[kt]
    if xbar is None:
        xbar = torch.empty(p + 1, dtype=torch.int64, device=A.device)
    if ybar is None:
        ybar = torch.empty(p + 1, dtype=torch.int64, device=A.device)
    code = load().tm_cross_ranks(_kt(kt), _dev(A, "A", kd), A.numel(), _dev(B, "B", kd), B.numel(), p,
                                 _dev(xbar, "xbar", (torch.int64,)), _dev(ybar, "ybar", (torch.int64,)),
                                 _stream(stream))
    _check(code, "tm_cross_ranks")
    return xbar, ybar


def tm_tile_record_bytes() -> int:
    return int(load().tm_tile_record_bytes())


def tm_merge_tile_cap(n: int, m: int, p: int) -> int:
    return int(load().tm_merge_tile_cap(n, m, p))


def tm_plan_tile_count(n: int, m: int, p: int) -> int:
    return int(load().tm_plan_tile_count(n, m, p))


@_on_stream
def tm_plan_subproblems(n: int, m: int, p: int, xbar, ybar, tiles=None, cfg=None, stream=None):
    """Steps 3-4 selection: tile records in merge-path order (uint8 tensor of
    room for 2p records; the first tm_plan_tile_count(n, m, p) are valid)."""
    if tiles is None:
        tiles = torch.empty(2 * p * tm_tile_record_bytes(), dtype=torch.uint8, device=xbar.device)
    code = load().tm_plan_subproblems(n, m, p, _dev(xbar, "xbar", (torch.int64,)), _dev(ybar, "ybar", (torch.int64,)),
                                      _dev(tiles, "tiles"), _cfg(cfg), _stream(stream))
    _check(code, "tm_plan_subproblems")
    return tiles


@_on_stream
def tm_merge_tiles(kt: str, A, Av, B, Bv, tiles, n_tiles: int, cap: int, C=None, Cv=None, control=None,
                   cfg=None, stream=None):
    """Steps 3-4 merges of planned tiles; returns (C, Cv, control).  The
    status word is control[0:4]."""
    kd = TORCH_KEY_DTYPES[kt]
    n, m = A.numel(), B.numel()
    if C is None:
        C = torch.empty(n + m, dtype=A.dtype, device=A.device)
    if Cv is None and (Av is not None or Bv is not None):
        Cv = torch.empty(n + m, dtype=(Av if Av is not None else Bv).dtype, device=A.device)
    if control is None:
        control = torch.zeros(256, dtype=torch.uint8, device=A.device)
    cfg = _payload_cfg(cfg, Av, Bv, Cv)
    P = ANY_PAYLOAD_DTYPES
    code = load().tm_merge_tiles(_kt(kt), _dev(A, "A", kd), _dev(Av, "Av", P), n, _dev(B, "B", kd), _dev(Bv, "Bv", P),
                                 m, _dev(tiles, "tiles"), n_tiles, cap, _dev(C, "C", kd), _dev(Cv, "Cv", P),
                                 _dev(control, "control"), _cfg(cfg), _stream(stream))
    _check(code, "tm_merge_tiles")
    return C, Cv, control


@_on_stream
def tm_rank_search(kt: str, kind: str, q, X, out=None, stream=None):
    """out[k] = rank_low(q[k], X) (kind 'low') or rank_high(q[k], X) ('high')."""
    kd = TORCH_KEY_DTYPES[kt]
    if out is None:
        out = torch.empty(q.numel(), dtype=torch.int64, device=q.device)
    code = load().tm_rank_search(_kt(kt), {"low": 0, "high": 1}[kind], _dev(q, "q", kd), q.numel(),
                                 _dev(X, "X", kd), X.numel(), _dev(out, "out", (torch.int64,)),
                                 _stream(stream))
    _check(code, "tm_rank_search")
    return out


@_on_stream
def tm_subproblems(n: int, m: int, p: int, xbar, ybar, table=None, stream=None):
    """Device-computed subproblem table, int64 (2p, 4): a0, a1, b0, b1."""
    if table is None:
        table = torch.empty((2 * p, 4), dtype=torch.int64, device=xbar.device)
    code = load().tm_subproblems(n, m, p, _dev(xbar, "xbar", (torch.int64,)), _dev(ybar, "ybar", (torch.int64,)),
                                 _dev(table, "table", (torch.int64,)), _stream(stream))
    _check(code, "tm_subproblems")
    return table


def tm_read_status(status, stream=None) -> int:
    """Synchronises the stream and returns the device status word (0 = ok)."""
    return int(load().tm_read_status(_dev(status, "status"), _stream(stream)))


PHASES = ("search", "barrier1", "select", "barrier2", "merge", "total")


def tm_merge_phase_times(workspace, n: int, m: int, cfg, stream=None) -> dict:
    """Phase times (microseconds) of the last traced fused launch of tm_merge
    on `workspace` (cfg with trace = 1, same n, m, cfg)."""
    out = (ctypes.c_double * 6)()
    code = load().tm_merge_phase_times(_dev(workspace, "workspace", (torch.uint8,)), n, m, _cfg(cfg),
                                       ctypes.cast(out, ctypes.c_void_p), _stream(stream))
    _check(code, "tm_merge_phase_times")
    return dict(zip(PHASES, list(out)))


TRACE_SLOTS = ("entry", "searched", "barrier", "selected", "selected2", "merged", "first_tile", "tiles")


def tm_merge_trace(workspace, n: int, m: int, cfg, stream=None) -> np.ndarray:
    """Per-CTA stamps of the last traced fused launch of tm_merge on
    `workspace` (cfg with trace = 1, same n, m, cfg): uint64 array (CTAs, 8),
    columns TRACE_SLOTS (%globaltimer nanoseconds, then the tile count)."""
    ctas = ctypes.c_int64(0)
    wp = _dev(workspace, "workspace", (torch.uint8,))
    load().tm_merge_trace(wp, n, m, _cfg(cfg), None, 0, ctypes.byref(ctas), _stream(stream))   # the CTA count
    out = np.zeros((max(ctas.value, 0), len(TRACE_SLOTS)), dtype=np.uint64)
    code = load().tm_merge_trace(wp, n, m, _cfg(cfg), out.ctypes.data_as(ctypes.c_void_p), out.size,
                                 ctypes.byref(ctas), _stream(stream))
    _check(code, "tm_merge_trace")
    return out


def tm_merge_noalloc(kt: str, A, Av, B, Bv, C, Cv, status=None, cfg=None, stream=None):
    """tm_merge without a workspace: the library keeps the cross ranks in its
    own built-in device array, so the call itself allocates nothing.  C, Cv
    (and the optional int32 `status`) are outputs the caller provides.
    Calls share that array: keep them ordered on one stream."""
    kd = TORCH_KEY_DTYPES[kt]
    n, m = A.numel(), B.numel()
    if C.numel() != n + m or Cv.numel() != n + m or Av.numel() != n or Bv.numel() != m:
        raise ValueError("length mismatch")
    code = load().tm_merge_noalloc(_kt(kt), _dev(A, "A", kd), _dev(Av, "Av", PAYLOAD_DTYPES), n, _dev(B, "B", kd),
                                   _dev(Bv, "Bv", PAYLOAD_DTYPES), m, _dev(C, "C", kd), _dev(Cv, "Cv", PAYLOAD_DTYPES),
                                   None if status is None else _dev(status, "status", (torch.int32,)),
                                   _cfg(cfg), _stream(stream))
    _check(code, "tm_merge_noalloc")
    return C, Cv


# ---------------------------------------------------------------------------
# Many merges, merge sort, autotuner, graphs
# ---------------------------------------------------------------------------

def _cfg_dict(c: TmConfig) -> dict:
    return {f: int(getattr(c, f)) for f, _ in TmConfig._fields_}


def tm_merge_batched_workspace_size(num_pairs: int, total_a: int, total_b: int, cfg=None) -> int:
    return int(load().tm_merge_batched_workspace_size(num_pairs, total_a, total_b, _cfg(cfg)))


def _batched_args(kt, a_off, A, Av, b_off, B, Bv, C, Cv):
    kd = TORCH_KEY_DTYPES[kt]
    pairs = a_off.numel() - 1
    if b_off.numel() != pairs + 1:
        raise ValueError("offset arrays differ in length")
    ta, tb = A.numel(), B.numel()
    if C is None:
        C = torch.empty(ta + tb, dtype=A.dtype, device=A.device)
    if Cv is None and (Av is not None or Bv is not None):
        Cv = torch.empty(ta + tb, dtype=(Av if Av is not None else Bv).dtype, device=A.device)
    P = ANY_PAYLOAD_DTYPES
    args = (_kt(kt), pairs, _dev(a_off, "a_off", (torch.int64,)), _dev(A, "A", kd), _dev(Av, "Av", P), ta,
            _dev(b_off, "b_off", (torch.int64,)), _dev(B, "B", kd), _dev(Bv, "Bv", P), tb,
            _dev(C, "C", kd), _dev(Cv, "Cv", P))
    return args, C, Cv, pairs, ta, tb


@_on_stream
def tm_merge_batched(kt: str, a_off, A, Av, b_off, B, Bv, C=None, Cv=None, workspace=None, cfg=None,
                     stream=None):
    """Independent stable merges of CSR pairs; returns (C, Cv, workspace)."""
    args, C, Cv, pairs, ta, tb = _batched_args(kt, a_off, A, Av, b_off, B, Bv, C, Cv)
    cfg = _payload_cfg(cfg, Av, Bv, Cv)
    if workspace is None:
        workspace = new_workspace(tm_merge_batched_workspace_size(pairs, ta, tb, cfg), A.device)
    code = load().tm_merge_batched(*args, _dev(workspace, "workspace"), workspace.numel(), _cfg(cfg),
                                   _stream(stream))
    _check(code, "tm_merge_batched")
    return C, Cv, workspace


def tm_merge_sort_workspace_size(n: int, cfg=None) -> int:
    return int(load().tm_merge_sort_workspace_size(n, _cfg(cfg)))


@_on_stream
def tm_merge_sort(kt: str, keys, vals, tmp_keys=None, tmp_vals=None, workspace=None, cfg=None, stream=None):
    """Stable sort of (keys, vals) in place; returns (keys, vals, workspace)."""
    kd = TORCH_KEY_DTYPES[kt]
    n = keys.numel()
    if tmp_keys is None:
        tmp_keys = torch.empty_like(keys)
    if tmp_vals is None and vals is not None:    # vals None: keys-only sort
        tmp_vals = torch.empty_like(vals)
    cfg = _payload_cfg(cfg, vals, tmp_vals)
    if workspace is None:
        workspace = new_workspace(tm_merge_sort_workspace_size(n, cfg), keys.device)
    code = load().tm_merge_sort(_kt(kt), _dev(keys, "keys", kd), _dev(vals, "vals", ANY_PAYLOAD_DTYPES), n,
                                _dev(tmp_keys, "tmp_keys", kd), _dev(tmp_vals, "tmp_vals", ANY_PAYLOAD_DTYPES),
                                _dev(workspace, "workspace"), workspace.numel(), _cfg(cfg), _stream(stream))
    _check(code, "tm_merge_sort")
    return keys, vals, workspace


def _host_offsets(seg_offsets) -> np.ndarray:
    """Segment offsets as a contiguous host int64 array (list, numpy array or
    CPU tensor)."""
    if isinstance(seg_offsets, torch.Tensor):
        if seg_offsets.is_cuda:
            raise ValueError("seg_offsets are read on the host: pass a CPU tensor, list or numpy array")
        seg_offsets = seg_offsets.numpy()
    return np.ascontiguousarray(np.asarray(seg_offsets, dtype=np.int64))


def tm_merge_sort_segmented_workspace_size(n: int, seg_offsets, cfg=None) -> int:
    off = _host_offsets(seg_offsets)
    return int(load().tm_merge_sort_segmented_workspace_size(n, off.ctypes.data_as(ctypes.c_void_p),
                                                             len(off) - 1, _cfg(cfg)))


@_on_stream
def tm_merge_sort_segmented(kt: str, keys, vals, seg_offsets, tmp_keys=None, tmp_vals=None, workspace=None,
                            cfg=None, stream=None):
    """Stable sort of every segment [seg_offsets[q], seg_offsets[q+1]) of
    (keys, vals) in place; seg_offsets on the host.  Returns (keys, vals,
    workspace)."""
    kd = TORCH_KEY_DTYPES[kt]
    n = keys.numel()
    off = _host_offsets(seg_offsets)
    if tmp_keys is None:
        tmp_keys = torch.empty_like(keys)
    if tmp_vals is None and vals is not None:
        tmp_vals = torch.empty_like(vals)
    cfg = _payload_cfg(cfg, vals, tmp_vals)
    if workspace is None:
        size = tm_merge_sort_segmented_workspace_size(n, off, cfg)
        if size == 0:
            raise TmError(TM_ERR_INVALID, "tm_merge_sort_segmented_workspace_size")
        workspace = new_workspace(size, keys.device)
    P = ANY_PAYLOAD_DTYPES
    code = load().tm_merge_sort_segmented(_kt(kt), _dev(keys, "keys", kd), _dev(vals, "vals", P), n,
                                          off.ctypes.data_as(ctypes.c_void_p), len(off) - 1,
                                          _dev(tmp_keys, "tmp_keys", kd), _dev(tmp_vals, "tmp_vals", P),
                                          _dev(workspace, "workspace"), workspace.numel(), _cfg(cfg),
                                          _stream(stream))
    _check(code, "tm_merge_sort_segmented")
    return keys, vals, workspace


def tm_autotune_batched(kt: str, a_off, A, Av, b_off, B, Bv, C, Cv, workspace, stream=None) -> dict:
    args, C, Cv, pairs, ta, tb = _batched_args(kt, a_off, A, Av, b_off, B, Bv, C, Cv)
    best = _cfg_struct(_payload_cfg(None, Av, Bv, Cv))
    code = load().tm_autotune_batched(*args, _dev(workspace, "workspace"), workspace.numel(),
                                      ctypes.byref(best), _stream(stream))
    _check(code, "tm_autotune_batched")
    return _cfg_dict(best)


def tm_autotune_sort(kt: str, src_keys, src_vals, keys, vals, tmp_keys, tmp_vals, workspace, stream=None) -> dict:
    kd = TORCH_KEY_DTYPES[kt]
    best = _cfg_struct(_payload_cfg(None, src_vals, vals, tmp_vals))
    P = ANY_PAYLOAD_DTYPES
    code = load().tm_autotune_sort(_kt(kt), _dev(src_keys, "src_keys", kd), _dev(src_vals, "src_vals", P),
                                   src_keys.numel(), _dev(keys, "keys", kd), _dev(vals, "vals", P),
                                   _dev(tmp_keys, "tmp_keys", kd), _dev(tmp_vals, "tmp_vals", P),
                                   _dev(workspace, "workspace"), workspace.numel(), ctypes.byref(best),
                                   _stream(stream))
    _check(code, "tm_autotune_sort")
    return _cfg_dict(best)


def tm_autotune_clear() -> int:
    return int(load().tm_autotune_clear())


def tm_graph_capture_begin(stream):
    _check(load().tm_graph_capture_begin(_stream(stream)), "tm_graph_capture_begin")


def tm_graph_capture_end(stream):
    h = ctypes.c_void_p()
    _check(load().tm_graph_capture_end(_stream(stream), ctypes.byref(h)), "tm_graph_capture_end")
    return h


def tm_graph_launch(g, stream=None):
    _check(load().tm_graph_launch(g, _stream(stream)), "tm_graph_launch")


def tm_graph_destroy(g):
    load().tm_graph_destroy(g)


class Graph:
    """Captures the tm_* calls made inside `with Graph(stream) as g:` on
    `stream` (a non-default torch.cuda.Stream, made current in the block)
    into a CUDA graph; g.launch() replays them.  A Graph must not be
    destroyed while another capture runs on the same thread (that
    invalidates the capture): rebinding a name that holds the previous
    Graph in `with Graph(s) as g:` does exactly that, so keep it alive."""

    def __init__(self, stream):
        self.stream = stream
        self.handle = None

    def __enter__(self):
        self._ctx = torch.cuda.stream(self.stream)
        self._ctx.__enter__()
        tm_graph_capture_begin(self.stream)
        return self

    def __exit__(self, *exc):
        try:
            self.handle = tm_graph_capture_end(self.stream)
        finally:
            self._ctx.__exit__(*exc)

    def launch(self, stream=None):
        tm_graph_launch(self.handle, stream or self.stream)

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                tm_graph_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


# ---------------------------------------------------------------------------
# Learned cross-rank proposal
# ---------------------------------------------------------------------------

LEARNED_ADVANCE = 1


class CdfModel:
    """A learned CDF model in a device buffer (layout in include/tm.h)."""

    HEADER = [("S", "<i4", 0), ("H", "<i4", 4), ("eps", "<f4", 8), ("cur", "<i4", 12), ("N", "<i8", 16),
              ("fallbacks", "<u8", 24), ("learned", "<u8", 32), ("adam_steps", "<i8", 40), ("loss", "<f4", 48)]

    def __init__(self, segments: int, hidden: int, device):
        self.S, self.H = int(segments), int(hidden)
        nbytes = int(load().tm_cdf_model_bytes(self.S, self.H))
        if nbytes == 0:
            raise ValueError("bad model dimensions")
        self.buf = torch.zeros(nbytes, dtype=torch.uint8, device=device)
        self.P = 4 * self.H + 1

    def _p(self):
        return _dev(self.buf, "model")

    @_on_stream
    def init(self, base, init_params, stream=None):
        ip = init_params.to(device=self.buf.device, dtype=torch.float32).contiguous()
        _check(load().tm_cdf_init(self._p(), self.S, self.H, _dev(base, "base", (torch.float32,)), base.numel(),
                                  _dev(ip, "init_params"), _stream(stream)), "tm_cdf_init")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        return self

    @_on_stream
    def grad(self, q, labels, stream=None):
        g = torch.empty(self.P, dtype=torch.float32, device=self.buf.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.buf.device)
        _check(load().tm_cdf_grad(self._p(), self.S, self.H, _dev(q, "q", (torch.float32,)),
                                  _dev(labels, "labels", (torch.int64,)), q.numel(), _dev(g, "g"), _dev(loss, "loss"),
                                  _stream(stream)), "tm_cdf_grad")
        return g, loss

    @_on_stream
    def train(self, q, labels, steps: int, lr: float, stream=None):
        _check(load().tm_cdf_train(self._p(), self.S, self.H, _dev(q, "q", (torch.float32,)),
                                   _dev(labels, "labels", (torch.int64,)), q.numel(), int(steps), float(lr),
                                   _stream(stream)), "tm_cdf_train")

    @_on_stream
    def predict(self, q, stream=None):
        out = torch.empty(q.numel(), dtype=torch.float32, device=q.device)
        _check(load().tm_cdf_predict(self._p(), self.S, self.H, _dev(q, "q", (torch.float32,)), q.numel(),
                                     _dev(out, "pred"), _stream(stream)), "tm_cdf_predict")
        return out

    @_on_stream
    def calibrate(self, q, labels, stream=None):
        _check(load().tm_cdf_calibrate(self._p(), self.S, self.H, _dev(q, "q", (torch.float32,)),
                                       _dev(labels, "labels", (torch.int64,)), q.numel(), _stream(stream)),
               "tm_cdf_calibrate")

    def _section(self, idx: int, dtype, count: int):
        # sections after the 256-byte header, each 256-byte aligned: K, R0, R1, params, m, v, grad, eps_seg
        sizes = [(self.S + 1) * 4, (self.S + 1) * 8, (self.S + 1) * 8] + [self.P * 4] * 4 + [self.S * 4]
        off = 256 + sum((x + 255) // 256 * 256 for x in sizes[:idx])
        return self.buf[off:off + count * torch.tensor([], dtype=dtype).element_size()].view(dtype)

    def knots(self):
        return self._section(0, torch.float32, self.S + 1)

    def ranks(self, which: int):
        return self._section(1 + which, torch.int64, self.S + 1)

    def params(self):
        return self._section(3, torch.float32, self.P)

    def eps_segments(self):
        return self._section(7, torch.float32, self.S)

    def header(self) -> dict:
        import numpy as np
        raw = self.buf[:64].cpu().numpy()
        return {name: np.frombuffer(raw[off:off + np.dtype(dt).itemsize].tobytes(), dtype=dt)[0].item()
                for name, dt, off in self.HEADER}


@_on_stream
def tm_cross_ranks_learned(model: CdfModel, A, B, p: int, xbar=None, ybar=None, flags: int = 0, stream=None):
    if xbar is None:
        xbar = torch.empty(p + 1, dtype=torch.int64, device=A.device)
    if ybar is None:
        ybar = torch.empty(p + 1, dtype=torch.int64, device=A.device)
    _check(load().tm_cross_ranks_learned(model._p(), model.S, model.H, _dev(A, "A", (torch.float32,)), A.numel(),
                                         _dev(B, "B", (torch.float32,)), B.numel(), p,
                                         _dev(xbar, "xbar", (torch.int64,)), _dev(ybar, "ybar", (torch.int64,)),
                                         int(flags), _stream(stream)), "tm_cross_ranks_learned")
    return xbar, ybar


def tm_merge_learned(model: CdfModel, A, Av, B, Bv, C=None, Cv=None, workspace=None, cfg=None, flags: int = 0,
                     stream=None):
    n, m = A.numel(), B.numel()
    if C is None:
        C = torch.empty(n + m, dtype=torch.float32, device=A.device)
    if Cv is None and (Av is not None or Bv is not None):
        Cv = torch.empty(n + m, dtype=torch.int32, device=A.device)
    if workspace is None:
        workspace = new_workspace(tm_merge_workspace_size(n, m, cfg), A.device)
    _check(load().tm_merge_learned(model._p(), model.S, model.H, _dev(A, "A", (torch.float32,)), _dev(Av, "Av", PAYLOAD_DTYPES), n,
                                   _dev(B, "B", (torch.float32,)), _dev(Bv, "Bv", PAYLOAD_DTYPES), m,
                                   _dev(C, "C", (torch.float32,)), _dev(Cv, "Cv", PAYLOAD_DTYPES), _dev(workspace, "workspace"),
                                   workspace.numel(), _cfg(cfg), int(flags), _stream(stream)), "tm_merge_learned")
    return C, Cv, workspace
