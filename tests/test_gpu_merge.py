"""GPU parity of the single stable merge (Steps 1-4) against the CPU oracle.

Every comparison is bit-exact: keys and payloads (payload = source tag |
index, so equal keys must come out A first and in input order)."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1202_6575_gb300 import tm, workloads as W
from tests.helpers import to_np, vals_np, first_mismatch

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "figure1.json")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def gpu_merge_check(kt, A, Av, B, Bv, cfg=None, offset_a=0, offset_b=0, offset_c=0):
    """Runs tm_merge on the GPU (optionally on sub-views shifted by a few
    elements, to exercise unaligned starts) and compares with the oracle."""
    def shifted(t, off):
        if off == 0:
            return t.to(DEV)
        big = torch.empty(t.numel() + off, dtype=t.dtype, device=DEV)
        big[off:] = t.to(DEV)
        return big[off:]
    dA, dAv, dB, dBv = shifted(A, offset_a), shifted(Av, offset_a), shifted(B, offset_b), shifted(Bv, offset_b)
    n, m = A.numel(), B.numel()
    Cb = torch.empty(n + m + offset_c, dtype=A.dtype, device=DEV)
    Cvb = torch.empty(n + m + offset_c, dtype=torch.int32, device=DEV)
    C, Cv, ws = tm.tm_merge(kt, dA, dAv, dB, dBv, Cb[offset_c:], Cvb[offset_c:], cfg=cfg)
    assert tm.tm_read_status(ws) == 0
    K, V = oracle.merge_two_pointer(to_np(A, kt), vals_np(Av), to_np(B, kt), vals_np(Bv))
    ck, cv = to_np(C, kt), vals_np(Cv)
    assert first_mismatch(ck, K) is None, f"key mismatch at {first_mismatch(ck, K)}"
    assert first_mismatch(cv, V) is None, f"payload mismatch at {first_mismatch(cv, V)}"


def test_figure1_cross_ranks_and_subproblems():
    g = json.load(open(GOLDEN))
    A = torch.tensor(g["A"], dtype=torch.int32, device=DEV)
    B = torch.tensor(g["B"], dtype=torch.int32, device=DEV)
    p = g["p"]
    xbar, ybar = tm.tm_cross_ranks("u32", A, B, p)
    assert xbar.tolist() == g["xbar"] and ybar.tolist() == g["ybar"]
    table = tm.tm_subproblems(len(g["A"]), len(g["B"]), p, xbar, ybar).cpu().numpy()
    otable = oracle.subproblems(len(g["A"]), len(g["B"]), p, np.array(g["xbar"]), np.array(g["ybar"]))
    for k in range(2 * p):
        lo, hi, olo, ohi, c0, case = otable[k]
        a0, a1, b0, b1 = table[k]
        if k < p:
            assert (a0, a1, b0, b1) == (lo, hi, olo, ohi)
        else:
            assert (b0, b1, a0, a1) == (lo, hi, olo, ohi)
        assert a0 + b0 == c0
    Av = W.payload(0, len(g["A"]), "cpu")
    Bv = W.payload(1, len(g["B"]), "cpu")
    gpu_merge_check("u32", A.cpu(), Av, B.cpu(), Bv, cfg={"p": p, "threads": 128})


def test_subproblem_table_matches_five_cases_exhaustively():
    rng = np.random.default_rng(0)
    for trial in range(300):
        n, m = int(rng.integers(0, 40)), int(rng.integers(0, 40))
        p = int(rng.integers(1, 14))
        alpha = int(rng.choice([1, 3, 30]))
        A = np.sort(rng.integers(0, alpha, n)).astype(np.uint32)
        B = np.sort(rng.integers(0, alpha, m)).astype(np.uint32)
        xb_o, yb_o = oracle.cross_ranks(A, B, p)
        dA = torch.from_numpy(A.view(np.int32)).to(DEV)
        dB = torch.from_numpy(B.view(np.int32)).to(DEV)
        xbar, ybar = tm.tm_cross_ranks("u32", dA, dB, p)
        assert xbar.cpu().numpy().tolist() == xb_o.tolist()
        assert ybar.cpu().numpy().tolist() == yb_o.tolist()
        table = tm.tm_subproblems(n, m, p, xbar, ybar).cpu().numpy()
        otable = oracle.subproblems(n, m, p, xb_o, yb_o)
        for k in range(2 * p):
            lo, hi, olo, ohi, c0, case = otable[k]
            a0, a1, b0, b1 = table[k]
            got = (a0, a1, b0, b1) if k < p else (b0, b1, a0, a1)
            assert got == (lo, hi, olo, ohi), (n, m, p, k, got, otable[k])


@pytest.mark.parametrize("split", [1, 2])
@pytest.mark.parametrize("kt", ["u32", "i32", "u64", "f32"])
@pytest.mark.parametrize("n,m", [(0, 0), (0, 7), (9, 0), (1, 1), (5, 3), (1000, 1), (4097, 4095),
                                 (30001, 20011), (100000, 3)])
def test_small_merges_all_key_types(kt, n, m, split):
    for alphabet in (None, 7):
        A, Av, B, Bv = W.small_merge(n, m, kt, seed=n * 31 + m, alphabet=alphabet)
        gpu_merge_check(kt, A, Av, B, Bv, cfg={"tile": 1024, "split": split})


@pytest.mark.parametrize("split,threads", [(1, 128), (1, 256), (1, 512), (2, 128), (2, 256)])
@pytest.mark.parametrize("tile", [256, 1000, 4096, 8192])
def test_tile_and_thread_shapes(threads, tile, split):
    A, Av, B, Bv = W.small_merge(70001, 50003, "u32", seed=tile + threads, alphabet=500)
    gpu_merge_check("u32", A, Av, B, Bv, cfg={"tile": tile, "threads": threads, "split": split})


@pytest.mark.parametrize("split,stages", [(1, 1), (1, 2), (1, 4), (2, 2), (2, 3), (2, 4)])
@pytest.mark.parametrize("kt", ["i32", "u64"])
def test_pipeline_depths(stages, split, kt):
    A, Av, B, Bv = W.small_merge(200003, 150001, kt, seed=stages * 7 + split, alphabet=300)
    gpu_merge_check(kt, A, Av, B, Bv, cfg={"tile": 2048, "stages": stages, "split": split})


@pytest.mark.parametrize("split", [1, 2])
@pytest.mark.parametrize("kt", ["u32", "u64"])
@pytest.mark.parametrize("offs", [(1, 0, 0), (0, 3, 1), (2, 1, 3), (3, 3, 2)])
def test_unaligned_starts(kt, offs, split):
    A, Av, B, Bv = W.small_merge(12345, 6789, kt, seed=sum(offs), alphabet=100)
    gpu_merge_check(kt, A, Av, B, Bv, cfg={"tile": 512, "split": split}, offset_a=offs[0], offset_b=offs[1],
                    offset_c=offs[2])


def test_explicit_p_larger_than_n():
    A, Av, B, Bv = W.small_merge(10, 300, "u32", seed=5, alphabet=20)
    gpu_merge_check("u32", A, Av, B, Bv, cfg={"p": 64})
    gpu_merge_check("u32", B, Bv, A, Av, cfg={"p": 64})


@pytest.mark.parametrize("split", [1, 2])
@pytest.mark.parametrize("dist", W.DIST_NAMES)
def test_distributions_small(dist, split):
    for skewed in (False, True):
        A, Av, B, Bv = W.large_merge(dist, skewed, "cpu", log2n=17, log2m_skewed=9)
        gpu_merge_check("i32", A, Av, B, Bv, cfg={"split": split})


@pytest.mark.parametrize("kt", ["u32", "i32", "u64", "f32"])
@pytest.mark.parametrize("n,m,p", [(1, 0, 1), (0, 5, 3), (7, 300, 64), (300, 7, 64), (5000, 3001, 8),
                                   (40000, 20000, 40), ((1 << 16) + 3, (1 << 15) - 1, 1024)])
def test_fused_launch_matches_separate_launches(kt, n, m, p):
    """Small merges run as one cooperative launch (searches, grid barrier,
    selection, merge); cfg unfused = 1 forces the separate launches.  Both
    must give the oracle's merge."""
    A, Av, B, Bv = W.small_merge(n, m, kt, seed=n + 7 * m + p, alphabet=50)
    gpu_merge_check(kt, A, Av, B, Bv, cfg={"p": p})
    gpu_merge_check(kt, A, Av, B, Bv, cfg={"p": p, "unfused": 1})


@pytest.mark.parametrize("kt,log2n,p", [("u64", 20, 1024), ("i32", 20, 1024), ("f32", 24, 16384)])
def test_fused_launch_full_tiles(kt, log2n, p):
    """Subproblems up to 2048 elements (the 17-element runs of the fused
    kernel) and the largest p the fused launch takes."""
    n = 1 << log2n
    A, Av, B, Bv = W.small_merge(n, n, kt, seed=log2n + p, alphabet=1 << 20)
    gpu_merge_check(kt, A, Av, B, Bv, cfg={"p": p})


@pytest.mark.parametrize("kt", ["u32", "i32", "u64", "f32"])
@pytest.mark.parametrize("n,m,cfg", [(5000, 3001, {"p": 8}), (200003, 150001, None),
                                     (70001, 50003, {"tile": 4096, "threads": 256}), (0, 9, None)])
def test_keys_only_merge(kt, n, m, cfg):
    """Payload pointers NULL: keys alone are merged (fused and separate
    launches, several tile shapes); the keys equal the oracle's."""
    A, Av, B, Bv = W.small_merge(n, m, kt, seed=n + m, alphabet=300)
    C, Cv, ws = tm.tm_merge(kt, A.to(DEV), None, B.to(DEV), None, cfg=cfg)
    assert Cv is None and tm.tm_read_status(ws) == 0
    K, _ = oracle.merge_two_pointer(to_np(A, kt), vals_np(Av), to_np(B, kt), vals_np(Bv))
    assert first_mismatch(to_np(C, kt), K) is None


@pytest.mark.parametrize("kt", ["u32", "i32", "u64", "f32"])
@pytest.mark.parametrize("n,m,alphabet", [(1 << 25, (1 << 25) + 17, 300), ((1 << 25) - 5, 1 << 25, None),
                                          (40_000_000, 3, None)])
def test_keys_only_merge_beyond_the_fused_range(kt, n, m, alphabet):
    """Keys-only merges above the fused launch's range with the default
    configuration take 8192-element tiles and 256 consumer threads (fewer
    blocks than the default sizing, which the workspace covers); every key
    equals the oracle's merge."""
    A, Av, B, Bv = W.small_merge(n, m, kt, seed=n + m, alphabet=alphabet, device=DEV)
    ws = tm.new_workspace(tm.tm_merge_workspace_size(n, m), DEV)
    C, Cv, ws = tm.tm_merge(kt, A, None, B, None, workspace=ws)
    assert Cv is None and tm.tm_read_status(ws) == 0
    K, _ = oracle.merge_two_pointer(to_np(A, kt), vals_np(Av), to_np(B, kt), vals_np(Bv))
    assert first_mismatch(to_np(C, kt), K) is None


@pytest.mark.parametrize("n,m", [(8191, 8193), (100003, 77777), (1 << 17, 5)])
def test_keys_only_merge_wide_tiles(n, m):
    """The keys-only large-merge configuration (tile 8192, 256 threads) set
    explicitly, at sizes with ragged tiles."""
    A, Av, B, Bv = W.small_merge(n, m, "u64", seed=n, alphabet=500)
    C, Cv, ws = tm.tm_merge("u64", A.to(DEV), None, B.to(DEV), None, cfg={"tile": 8192, "threads": 256})
    assert Cv is None and tm.tm_read_status(ws) == 0
    K, _ = oracle.merge_two_pointer(to_np(A, "u64"), vals_np(Av), to_np(B, "u64"), vals_np(Bv))
    assert first_mismatch(to_np(C, "u64"), K) is None


@pytest.mark.parametrize("kt", ["u32", "i32", "u64", "f32"])
@pytest.mark.parametrize("n,m,tile", [(0, 5, 64), (7, 0, 64), (1, 1, 64), (5000, 3001, 256),
                                      (100003, 77777, 2048), (1 << 16, 3, 1000), (3, 1 << 16, 4096)])
def test_equal_output_partition_ablation(kt, n, m, tile):
    """partition = TM_PARTITION_DIAGONALS (equal output ranges, the ablation
    against the paper's blocks) gives the same merge."""
    A, Av, B, Bv = W.small_merge(n, m, kt, seed=n + 3 * m + tile, alphabet=40)
    gpu_merge_check(kt, A, Av, B, Bv, cfg={"tile": tile, "partition": 1})


def test_fused_launch_in_cuda_graph_replayed():
    A, Av, B, Bv = W.small_merge(60000, 45001, "u32", seed=11, alphabet=1000)
    d = [t.to(DEV) for t in (A, Av, B, Bv)]
    cfg = {"p": 512}
    C = torch.empty(A.numel() + B.numel(), dtype=A.dtype, device=DEV)
    Cv = torch.empty_like(C, dtype=torch.int32)
    ws = tm.new_workspace(tm.tm_merge_workspace_size(A.numel(), B.numel(), cfg), DEV)
    s = torch.cuda.Stream()
    tm.tm_merge("u32", *d, C, Cv, ws, cfg=cfg, stream=s)
    s.synchronize()
    g = tm.Graph(s)
    with g:
        tm.tm_merge("u32", *d, C, Cv, ws, cfg=cfg, stream=s)
    K, V = oracle.merge_two_pointer(to_np(A, "u32"), vals_np(Av), to_np(B, "u32"), vals_np(Bv))
    for _ in range(2):
        C.fill_(-1)
        Cv.fill_(-1)
        torch.cuda.synchronize()
        g.launch()
        s.synchronize()
        assert tm.tm_read_status(ws, stream=s) == 0
        assert first_mismatch(to_np(C, "u32"), K) is None and first_mismatch(vals_np(Cv), V) is None


def test_single_merge_1m_p1024():
    """n = 2**20, m = 2**19 u32 keys in [0, 2**16), p = 1024."""
    A, Av, B, Bv = W.single_merge_1m(DEV)
    p = 1024
    xbar, ybar = tm.tm_cross_ranks("u32", A, B, p)
    xo, yo = oracle.cross_ranks(to_np(A, "u32"), to_np(B, "u32"), p)
    assert np.array_equal(xbar.cpu().numpy(), xo) and np.array_equal(ybar.cpu().numpy(), yo)
    gpu_merge_check("u32", A.cpu(), Av.cpu(), B.cpu(), Bv.cpu(), cfg={"p": p})


def test_three_phases_match_oracle_table():
    """tm_cross_ranks -> tm_plan_subproblems -> tm_merge_tiles.  The tile
    records (merge-path order) must be the oracle's five-case subproblems
    of the non-empty blocks, sorted by output offset."""
    rng = np.random.default_rng(2)
    for n, m, p in ((5000, 3000, 7), (40000, 1, 40), (1, 9000, 5), (30000, 30000, 64), (10, 300, 64)):
        A = np.sort(rng.integers(0, 200, n)).astype(np.uint32)
        B = np.sort(rng.integers(0, 200, m)).astype(np.uint32)
        dA = torch.from_numpy(A.view(np.int32)).to(DEV)
        dB = torch.from_numpy(B.view(np.int32)).to(DEV)
        Av = W.payload(0, n, DEV)
        Bv = W.payload(1, m, DEV)
        xbar, ybar = tm.tm_cross_ranks("u32", dA, dB, p)
        tiles = tm.tm_plan_subproblems(n, m, p, xbar, ybar)
        count = tm.tm_plan_tile_count(n, m, p)
        rec = tiles.view(torch.int64).view(2 * p, 6)[:count].cpu().numpy()
        otable = oracle.subproblems(n, m, p, xbar.cpu().numpy(), ybar.cpu().numpy())
        expect = []
        for k in range(2 * p):
            lo, hi, olo, ohi, oc0, case = otable[k]
            if hi == lo and ohi == olo:
                continue
            a = (lo, hi, olo, ohi) if k < p else (olo, ohi, lo, hi)
            expect.append((oc0, a[0], a[1] - a[0], a[2], a[3] - a[2]))
        expect.sort()
        got = [(int(r[2]), int(r[0]), int(r[3] & 0xffffffff), int(r[1]), int(r[3] >> 32)) for r in rec]
        assert got == expect, (n, m, p)
        cap = tm.tm_merge_tile_cap(n, m, p)
        C, Cv, control = tm.tm_merge_tiles("u32", dA, Av, dB, Bv, tiles, count, cap)
        assert tm.tm_read_status(control) == 0
        K, V = oracle.merge_two_pointer(A, vals_np(Av), B, vals_np(Bv))
        assert np.array_equal(to_np(C, "u32"), K) and np.array_equal(vals_np(Cv), V)


def test_rank_search_against_oracle():
    rng = np.random.default_rng(7)
    X = np.sort(rng.integers(0, 1000, 50000)).astype(np.uint32)
    q = rng.integers(0, 1100, 3000).astype(np.uint32)
    dX = torch.from_numpy(X.view(np.int32)).to(DEV)
    dq = torch.from_numpy(q.view(np.int32)).to(DEV)
    lo = tm.tm_rank_search("u32", "low", dq, dX).cpu().numpy()
    hi = tm.tm_rank_search("u32", "high", dq, dX).cpu().numpy()
    assert lo.tolist() == [oracle.rank_low(v, X) for v in q]
    assert hi.tolist() == [oracle.rank_high(v, X) for v in q]


@pytest.mark.parametrize("dist", W.DIST_NAMES)
@pytest.mark.parametrize("skewed", [False, True])
def test_large_merge_full_size(dist, skewed):
    """n = m = 2**28 (or n = 2**28, m = 2**18) int32 keys, the default launch
    configuration the benchmark times; every output element compared."""
    A, Av, B, Bv = W.large_merge(dist, skewed, DEV)
    C, Cv, ws = tm.tm_merge("i32", A, Av, B, Bv)
    assert tm.tm_read_status(ws) == 0
    hA, hAv, hB, hBv = to_np(A, "i32"), vals_np(Av), to_np(B, "i32"), vals_np(Bv)
    del A, Av, B, Bv
    ck, cv = to_np(C, "i32"), vals_np(Cv)
    del C, Cv
    torch.cuda.empty_cache()
    K, V = oracle.merge_two_pointer(hA, hAv, hB, hBv)
    assert first_mismatch(ck, K) is None, f"key mismatch at {first_mismatch(ck, K)}"
    assert first_mismatch(cv, V) is None, f"payload mismatch at {first_mismatch(cv, V)}"


def test_traced_fused_launch_gives_phase_times_and_the_same_merge():
    """cfg trace = 1 records per-CTA phase stamps of the fused launch; the
    merge is unchanged and the phases add up to the kernel's time."""
    A, Av, B, Bv = W.single_merge_1m("cpu")
    cfg = {"p": 1024, "trace": 1}
    gpu_merge_check("u32", A, Av, B, Bv, cfg=cfg)
    n, m = A.numel(), B.numel()
    ws = tm.new_workspace(tm.tm_merge_workspace_size(n, m, cfg), DEV)
    d = [t.to(DEV) for t in (A, Av, B, Bv)]
    tm.tm_merge("u32", *d, None, None, ws, cfg=cfg)
    ph = tm.tm_merge_phase_times(ws, n, m, cfg)
    assert all(v >= 0 for v in ph.values())
    assert ph["merge"] > 0 and ph["search"] > 0
    assert abs(sum(ph[k] for k in tm.PHASES[:5]) - ph["total"]) < 1e-6 * max(1.0, ph["total"]) + 1e-3
    # the per-CTA stamps behind the phases: ordered within each CTA, the
    # phase ends are the last CTAs' stamps, and the packed tiles hold every
    # record (one or more each; this workload's records average 768
    # elements, so a tile of at most 2176 packs few of them)
    tr = tm.tm_merge_trace(ws, n, m, cfg).astype(np.int64)
    assert tr.shape[1] == len(tm.TRACE_SLOTS) and tr.shape[0] >= 1
    assert np.all(tr[:, 1] >= tr[:, 0]) and np.all(tr[:, 2] >= tr[:, 1]) and np.all(tr[:, 5] >= tr[:, 2])
    t0 = tr[:, 0].min()
    assert abs((tr[:, 5].max() - t0) / 1e3 - ph["total"]) < 1e-3
    assert abs((tr[:, 1].max() - t0) / 1e3 - ph["search"]) < 1e-3
    R = tm.tm_plan_tile_count(n, m, 1024)
    assert R // 4 <= tr[:, 7].sum() <= R and tr[:, 7].min() >= 0
    # a separate-launch call records no trace
    cfg_u = {"p": 1024, "trace": 1, "unfused": 1}
    tm.tm_merge("u32", *d, None, None, ws, cfg=cfg_u)
    with pytest.raises(tm.TmError):
        tm.tm_merge_phase_times(ws, n, m, cfg_u)
