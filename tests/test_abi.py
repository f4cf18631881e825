"""The C-ABI library loads and exports every symbol include/tm.h declares;
host-side argument checks return their codes without touching a GPU."""
import ctypes
import os
import re

import pytest

import __graft_entry__  # noqa: F401  (puts the repo on sys.path)
from paper_1202_6575_gb300 import build, tm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"TM_API[^;(]*?\b(tm_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return tm.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "tm_merge" in names and len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    # and the binding knows every one of them
    assert set(names) <= set(tm.exported_symbols())


def test_status_strings(lib):
    assert tm.tm_status_str(0) == "ok"
    assert "workspace" in tm.tm_status_str(3)
    assert tm.tm_version() >= 1


def test_workspace_and_blocks_are_host_only(lib):
    assert tm.tm_merge_blocks(1 << 20, 1 << 19, {"p": 1024}) == 1024
    assert tm.tm_merge_blocks(0, 0) == 1
    assert tm.tm_merge_blocks(10000, 0, {"tile": 100}) == 100
    ws = tm.tm_merge_workspace_size(1 << 20, 1 << 19, {"p": 1024})
    assert ws >= 256 + 2 * 1025 * 8


def test_invalid_arguments_rejected_before_any_launch(lib):
    P = ctypes.c_void_p
    # negative length
    assert lib.tm_merge(0, None, None, -1, None, None, 0, None, None, None, 0, None, None) == tm.TM_ERR_INVALID
    # unknown key type
    assert lib.tm_merge(9, None, None, 0, None, None, 0, None, None, None, 0, None, None) == tm.TM_ERR_UNSUPPORTED
    # misaligned pointer
    assert lib.tm_merge(0, P(2), P(4), 3, P(8), P(8), 1, P(16), P(16), P(256), 1 << 20, None, None) == tm.TM_ERR_INVALID
    # missing workspace
    assert lib.tm_merge(0, P(16), P(16), 3, P(32), P(32), 1, P(64), P(64), None, 0, None, None) == tm.TM_ERR_WORKSPACE
    # workspace too small
    assert lib.tm_merge(0, P(16), P(16), 3, P(32), P(32), 1, P(64), P(64), P(256), 8, None, None) == tm.TM_ERR_WORKSPACE
    assert lib.tm_cross_ranks(0, P(16), 4, P(16), 4, 0, P(64), P(64), None) == tm.TM_ERR_INVALID
    assert lib.tm_merge_tiles(0, P(16), P(16), 4, P(16), P(16), 4, P(64), 1, 0, P(64), P(64), P(256), None, None) == tm.TM_ERR_INVALID
    assert lib.tm_plan_subproblems(4, 4, 0, P(64), P(64), P(64), None, None) == tm.TM_ERR_INVALID
    assert lib.tm_tile_record_bytes() == 48
    assert lib.tm_plan_tile_count(10, 3, 5) == 5 + 3
    assert lib.tm_merge_tile_cap(10, 7, 3) == 4 + 3
    assert lib.tm_rank_search(0, 2, P(16), 4, P(16), 4, P(64), None) == tm.TM_ERR_INVALID
    # payload pointers: all three or none (keys only); a mix is rejected
    assert lib.tm_merge(0, P(16), P(16), 3, P(32), None, 1, P(64), P(64), P(256), 1 << 20, None, None) == tm.TM_ERR_INVALID
    assert lib.tm_merge(0, P(16), None, 3, P(32), None, 1, P(64), P(64), P(256), 1 << 20, None, None) == tm.TM_ERR_INVALID
    assert lib.tm_merge(0, P(16), P(16), 3, P(32), P(32), 1, P(64), None, P(256), 1 << 20, None, None) == tm.TM_ERR_INVALID
    # keys only passes the argument checks (here: the missing workspace is reported next)
    assert lib.tm_merge(0, P(16), None, 3, P(32), None, 1, P(64), None, None, 0, None, None) == tm.TM_ERR_WORKSPACE
    # the allocation-free entry point has no keys-only form
    assert lib.tm_merge_noalloc(0, P(16), None, 3, P(32), None, 1, P(64), None, None, None, None) == \
        tm.TM_ERR_UNSUPPORTED


def test_invalid_arguments_of_the_batched_sort_graph_and_learned_calls(lib):
    """Every entry point's documented argument rules, on the host: each case
    returns its code before anything reaches the GPU (there is none here)."""
    P = ctypes.c_void_p
    INV, UNS, WS = tm.TM_ERR_INVALID, tm.TM_ERR_UNSUPPORTED, tm.TM_ERR_WORKSPACE
    off, k8, v4, ws = P(64), P(128), P(256), P(512)

    def batched(fn, pairs=2, aoff=off, ak=k8, av=v4, na=10, boff=off, bk=k8, bv=v4, nb=6, ck=k8, cv=v4,
                w=ws, wb=1 << 30, kt=2, last=None):
        args = [kt, pairs, aoff, ak, av, na, boff, bk, bv, nb, ck, cv, w, wb, last, None]
        return getattr(lib, fn)(*args)

    for fn in ("tm_merge_batched", "tm_autotune_batched"):
        assert batched(fn, pairs=-1) == INV
        assert batched(fn, na=-1) == INV
        assert batched(fn, kt=9) == UNS
        assert batched(fn, aoff=P(68)) == INV                    # offsets are int64
        assert batched(fn, bk=P(132)) == INV                     # u64 keys need 8-byte alignment
        assert batched(fn, av=None) == INV                       # payloads: all or none
        assert batched(fn, cv=None) == INV
        assert batched(fn, av=None, bv=None, cv=None, w=None) == WS   # keys only passes, then the workspace
        assert batched(fn, w=P(520)) == WS                       # workspace not 256-byte aligned
    assert batched("tm_merge_batched", wb=16) == WS
    assert lib.tm_merge_batched_workspace_size(-1, 0, 0, None) == 0
    assert lib.tm_merge_batched_workspace_size(4, 100, 100, None) > 0

    # tm_merge_sort(kt, keys, vals, n, tmp_keys, tmp_vals, ws, bytes, cfg, stream)
    assert lib.tm_merge_sort(2, k8, v4, -1, k8, v4, ws, 1 << 30, None, None) == INV
    assert lib.tm_merge_sort(9, k8, v4, 8, k8, v4, ws, 1 << 30, None, None) == UNS
    assert lib.tm_merge_sort(2, P(132), v4, 8, k8, v4, ws, 1 << 30, None, None) == INV
    assert lib.tm_merge_sort(2, k8, v4, 8, k8, None, ws, 1 << 30, None, None) == INV
    assert lib.tm_merge_sort(2, k8, None, 8, k8, None, None, 0, None, None) == WS
    assert lib.tm_merge_sort(2, k8, v4, 8, k8, v4, ws, 8, None, None) == WS
    assert lib.tm_merge_sort_workspace_size(-1, None) == 0
    # tm_autotune_sort(kt, src_k, src_v, n, keys, vals, tmp_k, tmp_v, ws, bytes, best, stream)
    assert lib.tm_autotune_sort(2, k8, v4, -1, k8, v4, k8, v4, ws, 1 << 30, None, None) == INV
    assert lib.tm_autotune_sort(9, k8, v4, 8, k8, v4, k8, v4, ws, 1 << 30, None, None) == UNS
    assert lib.tm_autotune_sort(2, k8, None, 8, k8, v4, k8, v4, ws, 1 << 30, None, None) == INV
    assert lib.tm_autotune_sort(2, k8, v4, 8, k8, v4, k8, v4, None, 0, None, None) == WS

    # graphs: the legacy stream cannot be captured; NULL handles
    h = ctypes.c_void_p()
    assert lib.tm_graph_capture_begin(None) == INV
    assert lib.tm_graph_capture_end(None, ctypes.byref(h)) == INV
    assert lib.tm_graph_launch(None, None) == INV
    lib.tm_graph_destroy(None)
    assert lib.tm_read_status(None, None) == INV

    # learned model: dimensions, alignment, counts
    assert lib.tm_cdf_model_bytes(1, 64) == 0 and lib.tm_cdf_model_bytes(4096, 0) == 0
    assert lib.tm_cdf_model_bytes(4096, 2048) == 0
    mb = lib.tm_cdf_model_bytes(4096, 64)
    assert mb > 0 and mb % 256 == 0
    model, q, lab, out = P(1 << 20), P(4096), P(8192), P(16384)
    assert lib.tm_cdf_init(P((1 << 20) + 64), 4096, 64, q, 100, q, None) == INV   # model not 256-aligned
    assert lib.tm_cdf_init(model, 4096, 64, q, 0, q, None) == INV
    assert lib.tm_cdf_grad(model, 4096, 64, q, lab, 0, out, out, None) == INV
    assert lib.tm_cdf_grad(model, 4096, 64, q, P(8196), 10, out, out, None) == INV   # labels are int64
    assert lib.tm_cdf_train(model, 4096, 64, q, lab, 10, -1, 1e-3, None) == INV
    assert lib.tm_cdf_predict(model, 4096, 64, q, -1, out, None) == INV
    assert lib.tm_cdf_predict(model, 4096, 64, q, 0, out, None) == tm.TM_OK          # nothing to do
    assert lib.tm_cdf_calibrate(model, 4096, 64, q, lab, 0, None) == INV
    # tm_cross_ranks_learned(model, S, H, a, n, b, m, p, xbar, ybar, flags, stream)
    assert lib.tm_cross_ranks_learned(model, 4096, 64, q, 100, q, 10, 0, out, out, 0, None) == INV
    assert lib.tm_cross_ranks_learned(model, 4096, 64, q, 0, q, 10, 4, out, out, 0, None) == INV
    assert lib.tm_cross_ranks_learned(model, 4096, 64, q, 100, q, 10, 4, P(16388), out, 0, None) == INV
    # tm_merge_learned(model, S, H, a, av, n, b, bv, m, c, cv, ws, bytes, cfg, flags, stream)
    assert lib.tm_merge_learned(model, 4096, 64, q, v4, 0, q, v4, 10, q, v4, ws, 1 << 30, None, 0, None) == INV
    assert lib.tm_merge_learned(model, 4096, 64, q, None, 100, q, v4, 10, q, v4, ws, 1 << 30, None, 0,
                                None) == INV
    assert lib.tm_merge_learned(model, 1, 64, q, v4, 100, q, v4, 10, q, v4, ws, 1 << 30, None, 0, None) == INV
    assert lib.tm_merge_learned(model, 4096, 64, P(4098), v4, 100, q, v4, 10, q, v4, ws, 1 << 30, None, 0,
                                None) == INV
    assert lib.tm_merge_learned(model, 4096, 64, q, v4, 100, q, v4, 10, q, v4, None, 0, None, 0, None) == WS
    # the allocation-free merge: lengths, key type, alignment
    assert lib.tm_merge_noalloc(0, k8, v4, -1, k8, v4, 1, k8, v4, None, None, None) == INV
    assert lib.tm_merge_noalloc(9, k8, v4, 1, k8, v4, 1, k8, v4, None, None, None) == UNS
    # phase times need a traced configuration and an output array
    out6 = (ctypes.c_double * 6)()
    assert lib.tm_merge_phase_times(P(256), 10, 10, None, ctypes.cast(out6, ctypes.c_void_p), None) == INV
    ct = tm.TmConfig(trace=1)
    assert lib.tm_merge_phase_times(P(256), 10, 10, ctypes.byref(ct), None, None) == INV
    assert lib.tm_merge_phase_times(P(8), 10, 10, ctypes.byref(ct), ctypes.cast(out6, ctypes.c_void_p), None) == INV
    # the per-CTA trace: a traced configuration, a count pointer, room or a count-only query
    cnt = ctypes.c_int64(-1)
    buf = (ctypes.c_uint64 * 16)()
    assert lib.tm_merge_trace(P(256), 10, 10, None, buf, 16, ctypes.byref(cnt), None) == INV
    assert lib.tm_merge_trace(P(256), 10, 10, ctypes.byref(ct), buf, 16, None, None) == INV
    assert lib.tm_merge_trace(P(256), 10, 10, ctypes.byref(ct), buf, -1, ctypes.byref(cnt), None) == INV
    assert lib.tm_merge_trace(P(256), 10, 10, ctypes.byref(ct), None, 16, ctypes.byref(cnt), None) == INV
    assert lib.tm_merge_trace(P(8), 10, 10, ctypes.byref(ct), buf, 16, ctypes.byref(cnt), None) == INV
    assert cnt.value == -1                                  # refused before anything was read
    # payload words: 4 or 8 bytes; 8-byte words need 8-byte alignment; the
    # learned and allocation-free calls take 4-byte words only
    c8 = tm.TmConfig(payload_bytes=8)
    v4only, v8 = P(260), P(264)                                # 4-byte but not 8-byte aligned; 8-byte aligned
    assert lib.tm_merge(0, k8, v4only, 10, k8, v8, 10, k8, v8, P(256), 1 << 20, ctypes.byref(c8), None) == INV
    assert lib.tm_merge(0, k8, v8, 10, k8, v8, 10, k8, v4only, P(256), 1 << 20, ctypes.byref(c8), None) == INV
    assert lib.tm_merge_batched(0, 1, P(16), k8, v4only, 10, P(16), k8, v8, 10, k8, v8, P(256), 1 << 30,
                                ctypes.byref(c8), None) == INV
    assert lib.tm_merge_sort(0, k8, v4only, 10, k8, v8, P(256), 1 << 30, ctypes.byref(c8), None) == INV
    assert lib.tm_merge_noalloc(0, k8, v8, 10, k8, v8, 10, k8, v8, None, ctypes.byref(c8), None) == UNS
    for bad in (3, 2, 16, -4):
        cb = tm.TmConfig(payload_bytes=bad)
        assert lib.tm_merge(0, k8, v4, 10, k8, v4, 10, k8, v4, P(256), 1 << 20, ctypes.byref(cb), None) == UNS
        assert lib.tm_merge_sort(0, k8, v4, 10, k8, v4, P(256), 1 << 30, ctypes.byref(cb), None) == UNS
    # runs merged per sort pass: 2 or 4 (0: the default)
    for ways in (1, 3, 8, -2):
        cw = tm.TmConfig(merge_ways=ways)
        assert lib.tm_merge_sort(0, k8, v4, 10, k8, v4, P(256), 1 << 30, ctypes.byref(cw), None) == UNS
    # configurations tm_merge refuses are refused here too (before any device work)
    for bad in ({"partition": tm.TM_PARTITION_DIAGONALS}, {"partition": 7}, {"threads": 64}, {"threads": 384}):
        c = tm.TmConfig(**bad)
        assert lib.tm_merge_noalloc(0, k8, v4, 10, k8, v4, 10, k8, v4, None, ctypes.byref(c), None) == UNS, bad


def test_binding_rejects_wrong_dtypes_before_the_device_check():
    import torch
    with pytest.raises(ValueError, match="dtype"):
        tm._dev(torch.zeros(4, dtype=torch.int64), "Av", tm.PAYLOAD_DTYPES)      # payloads are 32-bit words
    with pytest.raises(ValueError, match="dtype"):
        tm._dev(torch.zeros(4, dtype=torch.float32), "A", tm.TORCH_KEY_DTYPES["i32"])
    with pytest.raises(ValueError, match="contiguous"):
        tm._dev(torch.zeros(4, 2, dtype=torch.int32).t(), "A", tm.TORCH_KEY_DTYPES["i32"])
    with pytest.raises(ValueError, match="CUDA"):
        tm._dev(torch.zeros(4, dtype=torch.int32), "Av", tm.PAYLOAD_DTYPES)
    assert tm._dev(None, "Av", tm.PAYLOAD_DTYPES) == 0                           # keys-only call


def test_host_sizing_against_the_oracles_subproblems(lib):
    """tm_plan_tile_count is the number of non-empty blocks of A and B (one
    record each) and tm_merge_tile_cap bounds every subproblem the five
    cases produce (Section 2: one A-block piece plus one B-block piece),
    on random and tie-heavy inputs."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(21)
    for trial in range(300):
        n, m = int(rng.integers(0, 60)), int(rng.integers(0, 60))
        p = int(rng.integers(1, 20))
        alphabet = int(rng.choice([1, 2, 5, 1000]))
        A = np.sort(rng.integers(0, alphabet, size=n)).astype(np.uint32)
        B = np.sort(rng.integers(0, alphabet, size=m)).astype(np.uint32)
        nonempty = sum(oracle.block_start(n, p, i) < n for i in range(p)) + \
            sum(oracle.block_start(m, p, j) < m for j in range(p))
        assert lib.tm_plan_tile_count(n, m, p) == nonempty
        _, _, _, _, table = oracle.paper_merge(A, np.zeros(n, np.uint32), B, np.zeros(m, np.uint32), p)
        sizes = (table[:, 1] - table[:, 0]) + (table[:, 3] - table[:, 2])
        cap = lib.tm_merge_tile_cap(n, m, p)
        assert cap == -(-n // p) + -(-m // p)
        assert sizes.max(initial=0) <= cap and sizes.sum() == n + m


def test_header_is_c99_and_links_from_c(lib, tmp_path):
    """include/tm.h compiles as strict C99 and a C program links against
    libtm.so and calls its host-only entry points and argument checks."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "abi_c_client")
    libdir = os.path.dirname(tm.LIB_PATH)
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                           "-I" + os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "host", "abi_c_client.c"),
                           tm.LIB_PATH, "-Wl,-rpath," + libdir, "-o", exe])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip().endswith("all ok"), r.stdout + r.stderr


def test_binding_struct_matches_the_c_layout(tmp_path):
    """tm.TmConfig (ctypes) has the field names, offsets and sizes a C
    compiler gives struct tm_config of include/tm.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "abi_layout")
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Werror", "-I" + os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "host", "abi_layout.c"), "-o", exe])
    lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    c_fields = [ln.split() for ln in lines if ln and not ln.startswith("sizeof")]
    c_size = int(next(ln for ln in lines if ln.startswith("sizeof")).split()[1])
    py_fields = [(name, getattr(tm.TmConfig, name).offset, getattr(tm.TmConfig, name).size)
                 for name, _ in tm.TmConfig._fields_]
    assert [(n, int(o), int(s)) for n, o, s in c_fields] == py_fields
    assert c_size == ctypes.sizeof(tm.TmConfig)


def test_binding_derives_the_payload_width_from_the_tensors():
    import torch
    v32, v64 = torch.zeros(4, dtype=torch.int32), torch.zeros(4, dtype=torch.int64)
    assert tm._payload_cfg(None, v32, v32) is None
    assert tm._payload_cfg(None, v64, v64) == {"payload_bytes": 8}
    assert tm._payload_cfg({"p": 4}, v64, None) == {"p": 4, "payload_bytes": 8}
    assert tm._payload_cfg({"payload_bytes": 8}, v64) == {"payload_bytes": 8}
    assert tm._payload_cfg(tm.TmConfig(p=3), v64).payload_bytes == 8
    with pytest.raises(ValueError):
        tm._payload_cfg(None, v32, v64)
    with pytest.raises(ValueError):
        tm._payload_cfg({"payload_bytes": 4}, v64)
    with pytest.raises(ValueError):
        tm._payload_cfg(tm.TmConfig(payload_bytes=8), v32)


def test_segmented_sort_offsets_and_sizing_on_the_host(lib):
    """The segmented sort plans on the host: invalid offsets are refused
    before anything reaches a device, and the workspace grows with the
    number of rounds and pairs."""
    import numpy as np
    P = ctypes.c_void_p
    INV = tm.TM_ERR_INVALID

    def offs(v):
        a = np.ascontiguousarray(np.asarray(v, dtype=np.int64))
        return a, a.ctypes.data_as(P)

    for bad, n in (([1, 5], 5), ([0, 4], 5), ([0, 3, 2, 5], 5), ([0, 6], 5)):
        a, ptr = offs(bad)
        assert lib.tm_merge_sort_segmented_workspace_size(n, ptr, len(a) - 1, None) == 0
        assert lib.tm_merge_sort_segmented(0, P(256), P(512), n, ptr, len(a) - 1, P(768), P(1024), P(4096),
                                           1 << 30, None, None) == INV
    a1, p1 = offs([0, 1000, 1000, 5000])
    a2, p2 = offs([0, 1000, 1000, 1 << 20])
    s1 = lib.tm_merge_sort_segmented_workspace_size(5000, p1, 3, None)
    s2 = lib.tm_merge_sort_segmented_workspace_size(1 << 20, p2, 3, None)
    assert 0 < s1 < s2
    assert tm.tm_merge_sort_segmented_workspace_size(5000, [0, 1000, 1000, 5000]) == s1


def test_binding_runs_a_call_with_its_stream_current(monkeypatch):
    """A binding given `stream` (keyword or positional) runs with that
    stream current, so that the tensors it allocates belong to it; without
    one it runs on the caller's current stream."""
    entered = []

    class Ctx:
        def __init__(self, s):
            self.s = s

        def __enter__(self):
            entered.append(self.s)

        def __exit__(self, *exc):
            return False

    monkeypatch.setattr(tm.torch.cuda, "stream", Ctx)

    @tm._on_stream
    def call(a, b=None, stream=None):
        return (a, b, stream, list(entered))

    assert call(1) == (1, None, None, [])
    assert call(1, 2, stream="S1") == (1, 2, "S1", ["S1"])
    assert call(1, 2, "S2") == (1, 2, "S2", ["S1", "S2"])
    assert call(1, stream=None)[3] == ["S1", "S2"]

    class M:
        @tm._on_stream
        def meth(self, q, stream=None):
            return stream

    assert M().meth(3, "S3") == "S3" and entered[-1] == "S3"
    for f in (tm.tm_merge, tm.tm_merge_sort, tm.tm_merge_batched, tm.tm_merge_tiles, tm.tm_cross_ranks,
              tm.tm_merge_sort_segmented, tm.tm_cross_ranks_learned, tm.CdfModel.train):
        assert getattr(f, "__wrapped__", None) is not None, f.__name__
