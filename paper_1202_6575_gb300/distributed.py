"""Stable merge of arrays distributed over G ranks (the paper's closing
remark of Section 3: the merge on distributed memory, e.g. a BSP machine,
where dropping the merge of distinguished elements saves a communication
round; the paper leaves the details out, so the protocol below is this
library's reading).

Each rank holds one contiguous slice of A and one of B (any lengths, empty
allowed); globally A and B are sorted.  The protocol, one collective per
superstep:

1. allgather of the slice lengths (global offsets) and of the keys at the
   block starts x_i, y_j (Section 2's decomposition into p blocks) that fall
   in the rank's slices;
2. every rank counts, for every A-block start, the elements of its own B
   slice below it (rank_low) and, for every B-block start, the elements of
   its own A slice at or below it (rank_high); one allreduce (sum) gives
   the cross ranks xbar_i, ybar_j of Steps 1-2, since the slices are
   contiguous pieces of sorted arrays;
3. every rank plans all 2p subproblems (Steps 3-4, the five cases, by the
   library's plan kernel) in merge-path order and takes an equal share of
   them: rank g owns the contiguous merge-path segment from record
   g R / G to record (g + 1) R / G, i.e. A[a_lo, a_hi) and B[b_lo, b_hi)
   merging into C[a_lo + b_lo, a_hi + b_hi);
4. one all-to-all-v moves every rank's A and B segments (keys and
   payloads) to it; each piece is a contiguous part of one slice;
5. every rank merges its two segments (tm_merge) into its piece of C.

The result is C distributed in G contiguous pieces in rank order.
sort_distributed builds Section 3's merge sort on it: every rank sorts its
slice, then rounds of this merge join neighbouring groups of ranks.  The
collectives go through a small communicator interface: torch.distributed
(NCCL for device tensors, gloo for host tensors) or threads of one process
(for running the protocol of several ranks against one device).  The
per-rank computations go through an ops object; GpuOps runs them in this
library's kernels.
"""
from __future__ import annotations

import threading

import torch


def block_start(length: int, p: int, i: int) -> int:
    """x_i of Section 2: the first length mod p blocks hold one more element."""
    q, r = divmod(length, p)
    return i * (q + 1) if i < r else i * q + r


def first_block_at_or_after(length: int, p: int, k: int) -> int:
    """Smallest block index whose start is >= k (0 <= k <= length); for
    k = length the number of non-empty blocks, min(length, p)."""
    if k >= length:
        return min(length, p)
    q, r = divmod(length, p)
    head = r * (q + 1)
    j = k // (q + 1) if k < head else (k - head) // q + r
    return j if block_start(length, p, j) == k else j + 1


# ---------------------------------------------------------------------------
# Communicators
# ---------------------------------------------------------------------------

class TorchComm:
    """Collectives of a torch.distributed process group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def allgather(self, t: torch.Tensor) -> list:
        """The same-shape tensors of all ranks, in rank order."""
        out = [torch.empty_like(t) for _ in range(self.size)]
        self.dist.all_gather(out, t.contiguous(), group=self.group)
        return out

    def allreduce_sum(self, t: torch.Tensor) -> torch.Tensor:
        t = t.clone()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t

    def alltoallv(self, t: torch.Tensor, send: list, recv: list) -> torch.Tensor:
        """send[h] elements of t (in order) to rank h; recv[h] from rank h."""
        out = torch.empty(sum(recv), dtype=t.dtype, device=t.device)
        self.dist.all_to_all_single(out, t.contiguous(), recv, send, group=self.group)
        return out

    def split(self, groups: list) -> "TorchComm":
        """The communicator of this rank's group: groups partitions this
        communicator's ranks into lists (in rank order).  Collective: every
        process of the job calls it with the same groups."""
        base = (list(range(self.size)) if self.group is None
                else self.dist.get_process_group_ranks(self.group))
        mine = None
        for grp in groups:
            pg = self.dist.new_group(ranks=[base[r] for r in grp])
            if self.rank in grp:
                mine = TorchComm(pg)
        return mine


class ThreadHub:
    """Shared state of G ThreadComm ranks (one Python thread each)."""

    def __init__(self, size: int):
        self.size = size
        self.barrier = threading.Barrier(size)
        self.slots = [None] * size
        self._subs = {}
        self._lock = threading.Lock()

    def comm(self, rank: int) -> "ThreadComm":
        return ThreadComm(self, rank)

    def sub(self, key, size: int) -> "ThreadHub":
        """The hub of one group of a split (made by its first rank to ask)."""
        with self._lock:
            h = self._subs.get(key)
            if h is None:
                h = self._subs[key] = ThreadHub(size)
            return h

    def abort(self):
        """Releases every rank waiting here or in a group split from here."""
        self.barrier.abort()
        with self._lock:
            subs = list(self._subs.values())
        for h in subs:
            h.abort()


class ThreadComm:
    """Collectives among threads of one process: every call is a barrier
    that exchanges one value per rank."""

    def __init__(self, hub: ThreadHub, rank: int):
        self.hub, self.rank, self.size = hub, rank, hub.size
        self._splits = 0                              # splits made so far (the same on every rank)

    def _exchange(self, value):
        h = self.hub
        h.slots[self.rank] = value
        h.barrier.wait()
        got = list(h.slots)
        h.barrier.wait()                              # everyone has read before the next exchange
        return got

    def allgather(self, t: torch.Tensor) -> list:
        return [x.clone() for x in self._exchange(t)]

    def allreduce_sum(self, t: torch.Tensor) -> torch.Tensor:
        parts = self._exchange(t)
        out = parts[0].clone()
        for x in parts[1:]:
            out += x
        return out

    def alltoallv(self, t: torch.Tensor, send: list, recv: list) -> torch.Tensor:
        parts = self._exchange((t, list(send)))
        pieces = []
        for src, (tt, ss) in enumerate(parts):
            o = sum(ss[:self.rank])
            pieces.append(tt[o:o + ss[self.rank]])
            assert ss[self.rank] == recv[src], "send and receive counts disagree"
        return torch.cat(pieces) if pieces else t[:0]

    def split(self, groups: list) -> "ThreadComm":
        """The communicator of this rank's group (groups partitions the ranks)."""
        self._splits += 1
        for grp in groups:
            if self.rank in grp:
                return ThreadComm(self.hub.sub((self._splits, tuple(grp)), len(grp)), grp.index(self.rank))
        raise ValueError("rank in no group")


# ---------------------------------------------------------------------------
# Per-rank computations in the library's kernels
# ---------------------------------------------------------------------------

class GpuOps:
    """Steps of the protocol that touch data, on the device through the C
    ABI: block counts, rank searches, the subproblem plan, the local merge."""

    def __init__(self, kt: str, cfg=None):
        from . import tm
        self.tm = tm
        self.kt = kt
        self.cfg = cfg

    def blocks(self, n: int, m: int) -> int:
        return int(self.tm.tm_merge_blocks(n, m, self.cfg))

    def rank(self, kind: str, queries: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
        """rank_low ('low') or rank_high ('high') of every query in X (int64)."""
        if queries.numel() == 0:
            return torch.zeros(0, dtype=torch.int64, device=queries.device)
        if X.numel() == 0:
            return torch.zeros(queries.numel(), dtype=torch.int64, device=queries.device)
        return self.tm.tm_rank_search(self.kt, kind, queries, X)

    def chain_points(self, n: int, m: int, p: int, xbar: torch.Tensor, ybar: torch.Tensor) -> list:
        """Start points (a0, b0) of the subproblems in merge-path order, then
        (n, m): the plan kernel's records (first 16 bytes: int64 a0, b0)."""
        tm = self.tm
        count = tm.tm_plan_tile_count(n, m, p)
        rb = tm.tm_tile_record_bytes()
        tiles = torch.empty(max(1, 2 * p) * rb, dtype=torch.uint8, device=xbar.device)
        tm.tm_plan_subproblems(n, m, p, xbar, ybar, tiles)
        if count > 0:
            rec = tiles[:count * rb].view(torch.int64).view(count, rb // 8)[:, :2].cpu().tolist()
        else:
            rec = []
        return [tuple(r) for r in rec] + [(n, m)]

    def merge(self, A, Av, B, Bv):
        C, Cv, ws = self.tm.tm_merge(self.kt, A, Av, B, Bv, cfg=self.cfg)
        status = self.tm.tm_read_status(ws)
        if status != 0:
            raise RuntimeError(f"tm_merge: {self.tm.tm_status_str(status)}")
        return C, Cv

    def sort(self, K, Kv):
        """Stable sort of copies of (K, Kv) (tm_merge_sort)."""
        K = K.clone()
        Kv = None if Kv is None else Kv.clone()
        K, Kv, ws = self.tm.tm_merge_sort(self.kt, K, Kv, cfg=self.cfg)
        status = self.tm.tm_read_status(ws)
        if status != 0:
            raise RuntimeError(f"tm_merge_sort: {self.tm.tm_status_str(status)}")
        return K, Kv


# ---------------------------------------------------------------------------
# The protocol
# ---------------------------------------------------------------------------

def _overlap(lo: int, hi: int, s: int, e: int) -> int:
    return max(0, min(hi, e) - max(lo, s))


def merge_distributed(A: torch.Tensor, Av, B: torch.Tensor, Bv, comm, ops, p: int | None = None):
    """Stable merge of the distributed arrays whose slices this rank holds
    (A, Av: its slice of A and the payloads; B, Bv likewise; Av = Bv = None
    merges keys only).  Every rank calls it with the same p (None: the
    library's default for the global lengths).  Returns (C, Cv, c_lo, plan):
    this rank's piece of the merged output, which starts at global index
    c_lo, and the plan (global lengths, p, the G + 1 merge-path points that
    delimit the ranks' segments)."""
    G, g = comm.size, comm.rank
    dev = A.device
    # superstep 1: global offsets of every rank's slices
    lens = comm.allgather(torch.tensor([A.numel(), B.numel()], dtype=torch.int64, device=dev))
    lens = [tuple(int(v) for v in t.tolist()) for t in lens]
    offA = [sum(l[0] for l in lens[:h]) for h in range(G + 1)]
    offB = [sum(l[1] for l in lens[:h]) for h in range(G + 1)]
    n, m = offA[G], offB[G]
    if p is None:
        p = ops.blocks(n, m)
    # the block starts in this rank's slices (global block indices are
    # increasing with the rank, so the gathered keys come in block order)
    def starts_in(length, lo, hi):                    # blocks whose start lies in [lo, hi)
        return range(first_block_at_or_after(length, p, lo), first_block_at_or_after(length, p, hi))

    ia = starts_in(n, offA[g], offA[g + 1])
    jb = starts_in(m, offB[g], offB[g + 1])
    idx_a = torch.tensor([block_start(n, p, i) - offA[g] for i in ia], dtype=torch.int64, device=dev)
    idx_b = torch.tensor([block_start(m, p, j) - offB[g] for j in jb], dtype=torch.int64, device=dev)
    keys_a, keys_b = A[idx_a], B[idx_b]
    # allgather of variable counts: pad to the largest and send the counts
    na_all = [len(starts_in(n, offA[h], offA[h + 1])) for h in range(G)]
    nb_all = [len(starts_in(m, offB[h], offB[h + 1])) for h in range(G)]
    width = max(1, max(na_all), max(nb_all))
    pad = torch.zeros(2, width, dtype=A.dtype, device=dev)
    pad[0, :len(ia)] = keys_a
    pad[1, :len(jb)] = keys_b
    got = comm.allgather(pad)
    xa = torch.cat([got[h][0, :na_all[h]] for h in range(G)])      # keys of the non-empty A blocks
    yb = torch.cat([got[h][1, :nb_all[h]] for h in range(G)])
    # superstep 2: local counts, summed over the ranks = the cross ranks
    counts = torch.cat([ops.rank("low", xa, B), ops.rank("high", yb, A)])
    counts = comm.allreduce_sum(counts)
    xbar = torch.full((p + 1,), m, dtype=torch.int64, device=dev)  # empty blocks: the other length
    ybar = torch.full((p + 1,), n, dtype=torch.int64, device=dev)
    xbar[:xa.numel()] = counts[:xa.numel()]
    ybar[:yb.numel()] = counts[xa.numel():]
    # superstep 3: the plan, and this rank's share of the merge path
    points = ops.chain_points(n, m, p, xbar, ybar)
    R = len(points) - 1
    bounds = [points[(h * R) // G] for h in range(G)] + [points[R]]
    a_lo, b_lo = bounds[g]
    a_hi, b_hi = bounds[g + 1]
    # superstep 4: every piece to the rank whose segment contains it
    send_a = [_overlap(bounds[h][0], bounds[h + 1][0], offA[g], offA[g + 1]) for h in range(G)]
    send_b = [_overlap(bounds[h][1], bounds[h + 1][1], offB[g], offB[g + 1]) for h in range(G)]
    recv_a = [_overlap(a_lo, a_hi, offA[h], offA[h + 1]) for h in range(G)]
    recv_b = [_overlap(b_lo, b_hi, offB[h], offB[h + 1]) for h in range(G)]
    SA = comm.alltoallv(A, send_a, recv_a)
    SB = comm.alltoallv(B, send_b, recv_b)
    SAv = comm.alltoallv(Av, send_a, recv_a) if Av is not None else None
    SBv = comm.alltoallv(Bv, send_b, recv_b) if Bv is not None else None
    # the local merge of this rank's segment
    C, Cv = ops.merge(SA, SAv, SB, SBv)
    plan = {"n": n, "m": m, "p": p, "bounds": bounds, "records": R}
    return C, Cv, a_lo + b_lo, plan


def sort_distributed(K: torch.Tensor, Kv, comm, ops):
    """Stable sort of an array distributed over the G ranks of comm: rank g
    holds the contiguous slice (K, Kv) of it (any length, empty allowed; the
    array is the slices in rank order; Kv = None sorts keys only).  Section
    3's merge sort on distributed memory: every rank sorts its slice
    (ops.sort), then ceil(log2 G) rounds of merge_distributed; in round r
    the groups of 2^(r+1) neighbouring ranks merge the sorted arrays of their
    two halves (left half A, right half B, so that equal keys keep their
    global order), each group through its own communicator.  Returns (C, Cv,
    c_lo): this rank's piece of the sorted array, which starts at global
    index c_lo; the pieces are contiguous in rank order."""
    G, g = comm.size, comm.rank
    C, Cv = ops.sort(K, Kv)
    width = 1
    while width < G:
        groups = [list(range(s, min(G, s + 2 * width))) for s in range(0, G, 2 * width)]
        sub = comm.split(groups)
        if sub.size > width:                          # the group has a right half: merge the halves
            empty_v = None if Cv is None else Cv[:0]
            if g % (2 * width) < width:
                C, Cv, _, _ = merge_distributed(C, Cv, C[:0], empty_v, sub, ops)
            else:
                C, Cv, _, _ = merge_distributed(C[:0], empty_v, C, Cv, sub, ops)
        width *= 2
    lens = comm.allgather(torch.tensor([C.numel()], dtype=torch.int64, device=C.device))
    c_lo = sum(int(t.item()) for t in lens[:g])
    return C, Cv, c_lo
