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
