// Persistent, warp-specialised tile-merge engine shared by the single merge,
// the batched merge and the merge-sort passes.
//
// Work: a device array of tile descriptors, one per subproblem of Steps 3-4
// (an A range, a B range and the output offset they define).  Plan kernels
// write the descriptors; this kernel only moves and merges data.
//
// CTA = 1 producer warp + T consumer threads.
//  producer: pulls descriptors from a device work queue (atomicAdd, a few
//    tiles per grab), waits for a free input stage, writes the tile header,
//    and issues the bulk copies (cp.async.bulk, TMA engine) of the tile's
//    A keys, A payloads, B keys and B payloads on the stage's mbarrier.
//  consumers: wait for a full stage, re-split the tile among themselves by
//    the paper's rule (T blocks per piece, rank_low of each A-block start in
//    the B piece, rank_high of each B-block start in the A piece, then the 2T
//    sub-subproblems of the split-point form), merge serially into an output
//    buffer, release the input stage, and store the output with bulk copies
//    (16-byte aligned middle) plus plain stores for the ragged ends.
// Input stages and output buffers are multi-buffered, so the loads of later
// tiles and the stores of earlier ones overlap the merge of the current one.
#pragma once

#include "tm_common.cuh"

namespace pmerge {

// One subproblem: A[a0, a0+nA) and B[b0, b0+nB) merge into C[c0, c0+nA+nB).
// Plan kernels write the records in merge-path (chain) order, so that
// consecutive records are adjacent pieces of the merge path: their A ranges,
// B ranges and outputs are contiguous, and any run of them is itself a valid
// subproblem.
// `first` marks the first record of a merge (of a pair, in the batched
// form): records are never packed across it.
struct __align__(16) TileDesc {
    int64_t a0, b0, c0;
    int32_t nA, nB;
    int32_t first, pad0;
    int64_t pad1;
};
static_assert(sizeof(TileDesc) == 48, "descriptor layout");

// ceil(2^31 / d): floor(k / d) == (k * inv31(d)) >> 31 exactly for
// 0 <= k < 2^15 and 1 <= d <= 2^14 (the error term k*(M - 2^31/d)/2^31 stays
// below 2^-16 < 1/d).  Tiles hold at most 16386 elements, so every index
// and divisor of the in-CTA block arithmetic is in range.
__host__ __device__ __forceinline__ uint32_t inv31(uint32_t d) {
    return d ? (uint32_t)(((1ull << 31) + d - 1) / d) : 0u;
}
__device__ __forceinline__ int div_inv31(int k, uint32_t m) {
    return (int)(((uint64_t)(uint32_t)k * m) >> 31);
}

// The paper's block decomposition of `len` elements into T = 2^LOG_T blocks
// (first r blocks one longer), with the block-of-index rule by inverses.
template <int LOG_T>
struct BlockSplit {
    int len, q, r, head;
    uint32_t m1, m0;   // inverses of q + 1 and q
    __device__ __forceinline__ BlockSplit(int n, uint32_t inv_q1, uint32_t inv_q0)
        : len(n), q(n >> LOG_T), r(n & ((1 << LOG_T) - 1)), head(r * ((n >> LOG_T) + 1)), m1(inv_q1), m0(inv_q0) {}
    // x_i = i*q + min(i, r)  (= i*ceil for i < r, i*floor + r otherwise)
    __device__ __forceinline__ int start(int i) const { return i * q + min(i, r); }
    // block holding k (k = len -> T)
    __device__ __forceinline__ int of(int k) const {
        if (k >= len) return 1 << LOG_T;
        return (k < head) ? div_inv31(k, m1) : div_inv31(k - head, m0) + r;
    }
    // first block whose start is >= k
    __device__ __forceinline__ int first_at_or_after(int k) const {
        int j = of(k);
        return (start(j) == k) ? j : j + 1;
    }
};

// Named barrier among the consumer warps of one group (the producer never
// joins); group g uses barrier 1 + g.
__device__ __forceinline__ void consumer_sync(int nthreads, int id = 1) {
    asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(nthreads) : "memory");
}

// rank_low(x, X[0..len)) and rank_high(y, Y[0..len2)) in shared memory, as
// two interleaved branch-free bisections (power-of-two steps).
template <typename K>
__device__ __forceinline__ void rank_pair_smem(const K* X, int lenX, K x, int& rlow,
                                               const K* Y, int lenY, K y, int& rhigh) {
    int lo = 0, hi = 0;
    int mx = lenX > lenY ? lenX : lenY;
    if (mx > 0) {
        for (int step = 1 << (31 - __clz(mx)); step > 0; step >>= 1) {
            int a = lo + step, b = hi + step;
            if (a <= lenX && X[a - 1] < x) lo = a;
            if (b <= lenY && !(y < Y[b - 1])) hi = b;
        }
    }
    rlow = lo;
    rhigh = hi;
}

// Serial stable merge of sA[ia0..ia1) and sB[ib0..ib1) into sC from ia0 + ib0
// (B taken only when strictly smaller).  Reads at most one element past a
// range end, which lies inside the padded stage region.
template <typename K, typename V>
__device__ __forceinline__ void merge_run(const K* sAk, const V* sAv, int ia0, int ia1,
                                          const K* sBk, const V* sBv, int ib0, int ib1,
                                          K* sCk, V* sCv) {
    int i = ia0, j = ib0, o = ia0 + ib0;
    const int oend = ia1 + ib1;
    K ka = sAk[i];
    K kb = sBk[j];
#pragma unroll 2
    for (; o < oend; ++o) {
        const bool takeB = (j < ib1) && ((i >= ia1) || (kb < ka));
        const int idx = takeB ? j : i;
        const K* ks = takeB ? sBk : sAk;
        const V* vs = takeB ? sBv : sAv;
        sCk[o] = takeB ? kb : ka;
        sCv[o] = vs[idx];
        const K nxt = ks[idx + 1];
        if (takeB) { kb = nxt; ++j; } else { ka = nxt; ++i; }
    }
}

// Number of A elements among the first d outputs of the stable merge of
// sA[0..nA) and sB[0..nB): by the position formulas of Section 2 that is the
// i with B[d-i-1] < A[i] (A[i] lands at i + rank_low(A[i], B) >= d) and
// A[i-1] <= B[d-i] (B[d-i] lands at d-i + rank_high(B[d-i], A) >= d).
template <typename K>
__device__ __forceinline__ int corank_smem(const K* sA, int nA, const K* sB, int nB, int d) {
    int lo = d > nB ? d - nB : 0, hi = d < nA ? d : nA;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sB[d - mid - 1] < sA[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Stage layout
// ---------------------------------------------------------------------------
// Per input stage:  header (128 B) | keys region | payload region.
// A piece at the start of a region, B piece at a 16-byte boundary after it;
// each piece sits at the misalignment of its global source so that the
// aligned middle is one bulk copy.  Per output buffer: keys | payloads, at
// the misalignment of the global destination.  A keys-only launch (vsize 0)
// has no payload regions, so more CTAs fit on an SM.

struct EngineLayout {
    uint32_t stage_bytes, keys_off, vals_off;   // within a stage
    uint32_t out_bytes, out_vals_off;           // within an output buffer
    uint32_t split_off, bars_off;               // xs/ys, mbarriers
    uint32_t stages_off, outs_off, total;
};

__host__ __device__ inline uint32_t ru128(uint32_t x) { return (x + 127u) & ~127u; }

__host__ __device__ inline EngineLayout make_engine_layout(int cap, int ksize, int vsize, int T, int s_in,
                                                          int s_out) {
    EngineLayout L;
    uint32_t kreg = ru128((uint32_t)cap * ksize + 96);
    uint32_t vreg = vsize ? ru128((uint32_t)cap * vsize + 96) : 0u;
    L.keys_off = 128;
    L.vals_off = 128 + kreg;
    L.stage_bytes = 128 + kreg + vreg;
    L.out_vals_off = ru128((uint32_t)cap * ksize + 16);
    L.out_bytes = L.out_vals_off + (vsize ? ru128((uint32_t)cap * vsize + 16) : 0u);
    L.bars_off = 0;                                   // 2 * s_in mbarriers (<= 128 B)
    L.split_off = 128;
    uint32_t o = 128 + ru128(8u * (T + 1));
    L.stages_off = o;
    o += (uint32_t)s_in * L.stage_bytes;
    L.outs_off = o;
    o += (uint32_t)s_out * L.out_bytes;
    L.total = o;
    return L;
}

// Header the producer writes into a stage (read by the consumers).
struct StageHeader {
    int64_t c0;
    int32_t nA, nB;
    uint32_t mA1, mA0, mB1, mB0;
    uint32_t kA, kB, vA, vB;       // byte offsets of element 0 of each piece within its region
    int32_t end;                   // 1: no more tiles
};

struct EngineArgs {
    const TileDesc* desc;
    int64_t n_items;               // record count, or -1: read it from *n_items_dev
    const int64_t* n_items_dev;
    int64_t items_bound;           // upper bound of the record count (host side, for sizing)
    unsigned long long* queue;     // work-queue counter, zero at launch
    int32_t* status;
    const void* A; const void* Av; int64_t lenA;       // arrays the descriptors index; payload
    const void* B; const void* Bv; int64_t lenB;       // words of vbytes bytes (NULL: keys only)
    void* C; void* Cv;
    int vbytes;                                         // 4 or 8
    int cap;                       // max nA + nB of any tile
    int grab;                      // records per queue grab (<= 32)
    uint64_t wait_ns;              // limit of every mbarrier wait
    int drop_fill;                 // testing: fill index whose readiness signal is withheld (-1: none)
    EngineLayout lay;
    // Fused single merge (one cooperative launch): the kernel first computes
    // the cross ranks fx[0..p], fy[0..p] of A (lenA) and B (lenB), waits at a
    // grid barrier (gbar: arrival count, zero at launch), writes the records
    // of the 2p blocks into desc (Steps 3-4 selection), waits again, then
    // merges.
    int64_t* fx;
    int64_t* fy;
    int64_t fp;
    unsigned int* gbar;
    Blocks32 fbA, fbB;             // the block decompositions of A and B into fp blocks (n + fp < 2^32)
    // Profiling (nullptr = off): trace[0] = gridDim.x, then kTraceSlots
    // words per CTA from trace[kTraceSlots]: %globaltimer at kernel entry,
    // searches done, barrier passed, first subproblems selected (twice: the
    // launch has no second barrier), merges done, first tile landed; then
    // the number of tiles the CTA merged.
    uint64_t* trace;
};

constexpr int kTraceSlots = 8;

__device__ __forceinline__ void trace_stamp(const EngineArgs& g, int slot) {
    if (g.trace != nullptr && threadIdx.x == 0) {
        g.trace[(size_t)kTraceSlots * (blockIdx.x + 1) + slot] = global_timer_ns();
        if (slot == 0 && blockIdx.x == 0) g.trace[0] = gridDim.x;
    }
}

// Bulk-copy window of elements [lo, lo+cnt) of an array (base, len,
// element size E) into a region at byte offset `dst_off`: the region
// receives the 16-byte window starting at round_down(&X[lo], 16); the bytes
// [t0, t1) inside the array's own aligned span go by bulk copy, anything of
// [g0, g1) outside it (only next to the array's first or last 16 bytes) by
// plain loads.  Pass 0 does the plain loads and returns the bulk bytes in
// tx_bytes; pass 1 issues the bulk copy.  Returns the byte offset of X[lo]
// within the region.
__device__ __forceinline__ uint32_t stage_piece(uint8_t* region, uint32_t dst_off, const void* base,
                                                int64_t len, int64_t lo, int64_t cnt, uint32_t E,
                                                uint64_t* bar, uint32_t& tx_bytes, int pass) {
    uintptr_t b = reinterpret_cast<uintptr_t>(base);
    uintptr_t g0 = b + (uintptr_t)lo * E, g1 = g0 + (uintptr_t)cnt * E;
    uintptr_t w0 = g0 & ~(uintptr_t)15;
    uintptr_t lim0 = (b + 15) & ~(uintptr_t)15, lim1 = (b + (uintptr_t)len * E) & ~(uintptr_t)15;
    uintptr_t t0 = w0 > lim0 ? w0 : lim0;
    uintptr_t r1 = (g1 + 15) & ~(uintptr_t)15;
    uintptr_t t1 = r1 < lim1 ? r1 : lim1;
    uint8_t* dst = region + dst_off;
    if (cnt > 0) {
        if (t1 > t0) {
            if (pass == 1) bulk_g2s(dst + (t0 - w0), reinterpret_cast<const void*>(t0), (uint32_t)(t1 - t0), bar);
            else tx_bytes += (uint32_t)(t1 - t0);
        } else {
            t0 = t1 = g1;                         // no bulk part: all plain
        }
        if (pass == 0) {                          // plain loads of [g0, min(t0, g1)) and [max(t1, g0), g1)
            for (uintptr_t a = g0; a < g1 && a < t0; a += E) {
                if (E == 8) *reinterpret_cast<uint64_t*>(dst + (a - w0)) = *reinterpret_cast<const uint64_t*>(a);
                else        *reinterpret_cast<uint32_t*>(dst + (a - w0)) = *reinterpret_cast<const uint32_t*>(a);
            }
            for (uintptr_t a = (t1 > g0 ? t1 : g0); a < g1; a += E) {
                if (E == 8) *reinterpret_cast<uint64_t*>(dst + (a - w0)) = *reinterpret_cast<const uint64_t*>(a);
                else        *reinterpret_cast<uint32_t*>(dst + (a - w0)) = *reinterpret_cast<const uint32_t*>(a);
            }
        }
    }
    return dst_off + (uint32_t)(g0 - w0);
}

// Output of L elements at C[c0..): bulk store of the aligned middle (one
// thread) and plain stores of the ragged ends.  `buf` holds element 0 at
// byte offset (destination address & 15).
template <typename T>
__device__ __forceinline__ void store_out(const uint8_t* buf, const void* base, int64_t c0, int L,
                                          int tid, int nthreads, bool issuer) {
    const uintptr_t E = sizeof(T);
    uintptr_t g0 = reinterpret_cast<uintptr_t>(base) + (uintptr_t)c0 * E;
    uintptr_t g1 = g0 + (uintptr_t)L * E;
    uintptr_t m0 = (g0 + 15) & ~(uintptr_t)15, m1 = g1 & ~(uintptr_t)15;
    const uint8_t* src0 = buf + (g0 & 15);              // element 0 in the buffer
    if (m1 > m0) {
        if (issuer) bulk_s2g(reinterpret_cast<void*>(m0), src0 + (m0 - g0), (uint32_t)(m1 - m0));
        int nh = (int)((m0 - g0) / E), t0 = (int)((m1 - g0) / E);
        if (tid < nh) reinterpret_cast<T*>(g0)[tid] = reinterpret_cast<const T*>(src0)[tid];
        int e = t0 + tid;
        if (e < L) reinterpret_cast<T*>(g0)[e] = reinterpret_cast<const T*>(src0)[e];
    } else {
        for (int e = tid; e < L; e += nthreads) reinterpret_cast<T*>(g0)[e] = reinterpret_cast<const T*>(src0)[e];
    }
}

// Steps 3-4 selection of block k of a single merge (A-side block k for k < p,
// B-side block k - p otherwise): its subproblem from the five cases in
// split-point form, written as the record at its merge-path (chain) index.
// A-point P_A(i) has i A-points and first_block_at_or_after(m, p, xbar_i)
// B-points before it, and symmetrically for P_B(j), so the chain index is a
// sum of two O(1) terms.  Empty blocks (p above a length) write nothing; the
// non-empty records fill indices [0, min(p, n) + min(p, m)).
template <typename LoadX, typename LoadY>
__device__ __forceinline__ void plan_single_record(int64_t n, int64_t m, int64_t p, int64_t k, LoadX xb, LoadY yb,
                                                   TileDesc* desc) {
    const bool a_side = k < p;
    const int64_t pe = a_side ? k : k - p;
    if (a_side ? block_start<int64_t>(n, p, pe) >= n : block_start<int64_t>(m, p, pe) >= m) return;
    int64_t a0, a1, b0, b1;
    subproblem_of<int64_t>(a_side, pe, n, m, p, xb, yb, a0, a1, b0, b1);
    const int64_t chain = a_side ? pe + first_block_at_or_after<int64_t>(m, p, xb(pe))
                                 : pe + first_block_at_or_after<int64_t>(n, p, yb(pe));
    TileDesc d{};
    d.a0 = a0; d.b0 = b0; d.c0 = a0 + b0;
    d.nA = (int32_t)(a1 - a0); d.nB = (int32_t)(b1 - b0);
    d.first = chain == 0;
    desc[chain] = d;
}

// Rank of x in sorted X[0..len) by one warp: each round the 32 lanes probe
// 32 positions splitting the candidate range [lo, hi] into 33 parts, and
// the count of probes that lie before x (X sorted: a prefix of the lanes)
// keeps one part: ceil(log33(len + 1)) rounds of independent loads instead
// of ceil(log2(len + 1)) dependent probes.  HIGH: rank_high (elements <= x),
// else rank_low (elements < x).  Every lane returns the rank.  The part
// boundaries q_r = lo + ceil(r w / 33) in 32-bit arithmetic: with
// w = 33 u + v (0 <= v < 33), ceil(r w / 33) = r u + ceil(r v / 33), where
// r v < 33^2 keeps the division small.  len < 2^32.
__device__ __forceinline__ uint32_t part33(uint32_t r, uint32_t u, uint32_t v) {
    return r * u + (r * v + 32u) / 33u;
}

template <bool HIGH, typename K>
__device__ __forceinline__ int64_t warp_rank33(const K* __restrict__ X, uint32_t len, K x, int lane) {
    uint32_t lo = 0, hi = len;
    while (hi > lo) {
        const uint32_t w = hi - lo, u = w / 33u, v = w - 33u * (w / 33u);
        const uint32_t q = lo + part33((uint32_t)lane + 1u, u, v);     // in (lo, hi]
        const K val = __ldg(X + q - 1);
        const bool before = HIGH ? !(x < val) : (val < x);
        const int c = __popc(__ballot_sync(0xffffffffu, before));
        // probes 1..c lie before x: the rank is in [q_c, q_{c+1} - 1]
        const uint32_t qlo = c > 0 ? lo + part33((uint32_t)c, u, v) : lo;
        const uint32_t qhi = c < 32 ? lo + part33((uint32_t)c + 1u, u, v) - 1u : hi;
        lo = qlo;
        hi = qhi;
    }
    return (int64_t)lo;
}

// Fused single merge, Steps 1-2: the 2p + 1 cross ranks, one warp per
// search, strided over every warp of the grid (B-block starts first).
template <typename K>
__device__ __forceinline__ void fused_cross_ranks(const EngineArgs& g) {
    const K* A = static_cast<const K*>(g.A);
    const K* B = static_cast<const K*>(g.B);
    const int64_t n = g.lenA, m = g.lenB, p = g.fp;
    const int lane = threadIdx.x & 31;
    const int64_t wpc = blockDim.x >> 5;
    const int64_t stride = (int64_t)gridDim.x * wpc;
    for (int64_t t = (int64_t)blockIdx.x * wpc + (threadIdx.x >> 5); t <= 2 * p; t += stride) {
        if (t < p) {
            const int64_t yj = g.fbB.start(t);
            const int64_t r = (yj < m) ? warp_rank33<true, K>(A, (uint32_t)n, __ldg(B + yj), lane) : n;
            if (lane == 0) g.fy[t] = r;
        } else if (t < 2 * p) {
            const int64_t i = t - p;
            const int64_t xi = g.fbA.start(i);
            const int64_t r = (xi < n) ? warp_rank33<false, K>(B, (uint32_t)m, __ldg(A + xi), lane) : m;
            if (lane == 0) g.fx[i] = r;
        } else if (lane == 0) {
            g.fx[p] = m;
            g.fy[p] = n;
        }
    }
}

// Grid-wide barrier of a cooperative launch (every CTA resident).  bar counts
// arrivals over the whole launch (zero at launch): the k-th barrier of the
// launch waits until it reaches k * gridDim.x.  Thread 0 arrives with a
// release add after the CTA's barrier and polls with acquire loads (backing
// off 64 ns between polls), at most limit_ns of global time (then
// TM_ERR_TIMEOUT and false).  The same value for every thread of the CTA.
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned int k, uint64_t limit_ns, int32_t* status) {
    __shared__ int passed;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int target = k * gridDim.x;
        unsigned int v;
        asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(v) : "l"(bar) : "memory");
        int ok = 1;
        if (v + 1 < target) {
            const uint64_t t0 = global_timer_ns();
            for (;;) {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
                if (v >= target) break;
                if (global_timer_ns() - t0 > limit_ns) { ok = 0; set_status(status, TM_ERR_TIMEOUT); break; }
                __nanosleep(64);
            }
        }
        passed = ok;
    }
    __syncthreads();
    return passed != 0;
}

// In-CTA split of a staged tile among the consumer threads:
//   kSplitBlocks   - the paper's rule again: T blocks per piece, cross ranks
//                    of the block starts, 2T sub-subproblems, two per thread,
//                    merged into a separate output buffer;
//   kSplitDiagonal - equal output runs of VT elements (VT odd): thread t
//                    starts at the co-rank of output diagonal t*VT (the
//                    position formulas of Section 2) and merges VT elements
//                    into registers; the runs are then written back into the
//                    consumed input stage (odd VT: bank-conflict free) and
//                    stored from there.
enum { kSplitBlocks = 0, kSplitDiagonal = 1 };

// Stages one tile -- A[a0, a0+nA) and B[b0, b0+nB), output from c0 -- into
// input stage k % S_IN (the k-th fill of the CTA) once the consumers have
// freed it.  Lanes 0..3 copy the four pieces (A keys, A payloads, B keys, B
// payloads) in parallel; lane 0 writes the header and arms the stage's
// barrier.  Returns false when the wait for a free stage gave up
// (TM_ERR_TIMEOUT set); a tile over its capacity sets TM_ERR_BOUNDS and is
// skipped.  Advances k for every fill it takes.
template <typename K, typename V, int LOG_T, int S_IN, int SPLIT>
__device__ __forceinline__ bool stage_tile(const EngineArgs& g, uint8_t* smem, uint64_t* full, uint64_t* empty,
                                           int lane, int& k, int64_t a0, int64_t b0, int64_t c0, int nA, int nB) {
    if (nA + nB == 0) return true;
    if (nA < 0 || nB < 0 || nA + nB > g.cap) {
        if (lane == 0) set_status(g.status, TM_ERR_BOUNDS);
        return true;
    }
    const int s = k % S_IN;
    int free_ok = 1;
    if (lane == 0 && k >= S_IN) free_ok = mbar_wait_bounded(&empty[s], ((k / S_IN) & 1) ^ 1, g.wait_ns) ? 1 : 0;
    free_ok = __shfl_sync(0xffffffffu, free_ok, 0);
    if (!free_ok) {
        if (lane == 0) set_status(g.status, TM_ERR_TIMEOUT);
        return false;
    }
    if (k == g.drop_fill) {                           // testing: this stage never becomes ready
        ++k;
        return true;
    }
    uint8_t* st = smem + g.lay.stages_off + (uint32_t)s * g.lay.stage_bytes;
    // piece of this lane: 0 A keys, 1 A payloads, 2 B keys, 3 B payloads
    const bool isB = lane >= 2, isV = (lane & 1) != 0;
    const uint32_t E = isV ? (uint32_t)sizeof(V) : (uint32_t)sizeof(K);
    const void* pbase = isB ? (isV ? g.Bv : g.B) : (isV ? g.Av : g.A);
    // keys-only merge (no payload arrays): the payload pieces are empty
    const int64_t plen = isB ? g.lenB : g.lenA, plo = isB ? b0 : a0;
    const int64_t pcnt = (isV && g.Cv == nullptr) ? 0 : (isB ? nB : nA);
    uint8_t* region = st + (isV ? g.lay.vals_off : g.lay.keys_off);
    uint32_t dst_off = 0;
    if (isB) {   // after the A piece of the same region, on a 16-byte boundary
        const uintptr_t abase = reinterpret_cast<uintptr_t>(isV ? g.Av : g.A);
        const uint32_t aoff = (uint32_t)((abase + (uintptr_t)a0 * E) & 15);
        dst_off = (aoff + (uint32_t)nA * E + 31u) & ~15u;
    }
    uint32_t tx = 0, off = 0, inv = 0;
    if (lane < 4) {
        off = stage_piece(region, dst_off, pbase, plen, plo, pcnt, E, &full[s], tx, 0);
        if (SPLIT == kSplitBlocks) {                  // inverses of q+1 and q per piece length
            const uint32_t qn = (uint32_t)(isB ? nB : nA) >> LOG_T;
            inv = inv31(isV ? qn : qn + 1);
        }
    }
    tx += __shfl_xor_sync(0xffffffffu, tx, 1);
    tx += __shfl_xor_sync(0xffffffffu, tx, 2);
    const uint32_t oKA = __shfl_sync(0xffffffffu, off, 0), oVA = __shfl_sync(0xffffffffu, off, 1);
    const uint32_t oKB = __shfl_sync(0xffffffffu, off, 2), oVB = __shfl_sync(0xffffffffu, off, 3);
    const uint32_t mA1 = __shfl_sync(0xffffffffu, inv, 0), mA0 = __shfl_sync(0xffffffffu, inv, 1);
    const uint32_t mB1 = __shfl_sync(0xffffffffu, inv, 2), mB0 = __shfl_sync(0xffffffffu, inv, 3);
    __syncwarp();                                     // plain edge loads before the arrive
    if (lane == 0) {
        StageHeader* h = reinterpret_cast<StageHeader*>(st);
        h->c0 = c0; h->nA = nA; h->nB = nB;
        h->mA1 = mA1; h->mA0 = mA0; h->mB1 = mB1; h->mB0 = mB0;
        h->kA = oKA; h->vA = oVA; h->kB = oKB; h->vB = oVB;
        h->end = 0;
        mbar_arrive_expect_tx(&full[s], tx);
    }
    __syncwarp();
    uint32_t unused = 0;
    if (lane < 4) stage_piece(region, dst_off, pbase, plen, plo, pcnt, E, &full[s], unused, 1);
    ++k;
    return true;
}

// End markers for the consumers after the last fill (lane 0): one in each
// of the next NG fills, so that every consumer group (group j takes the
// fills j, j + NG, ...) finds one.
template <int S_IN, int NG = 1>
__device__ __forceinline__ void stage_end(const EngineArgs& g, uint8_t* smem, uint64_t* full, uint64_t* empty,
                                          int lane, int k) {
    if (lane != 0) return;
    for (int e = 0; e < NG; ++e, ++k) {
        const int s = k % S_IN;
        if (k >= S_IN && !mbar_wait_bounded(&empty[s], ((k / S_IN) & 1) ^ 1, g.wait_ns)) {
            set_status(g.status, TM_ERR_TIMEOUT);
            return;
        }
        StageHeader* h = reinterpret_cast<StageHeader*>(smem + g.lay.stages_off + (uint32_t)s * g.lay.stage_bytes);
        h->end = 1;
        mbar_arrive_expect_tx(&full[s], 0);
    }
}

// Producer warp: pulls tile records from the work queue and stages them.
// A grab of G consecutive records is packed greedily into tiles of at most
// `cap` elements (consecutive records are adjacent on the merge path).
template <typename K, typename V, int LOG_T, int S_IN, int SPLIT, int NG = 1>
__device__ __forceinline__ void engine_producer(const EngineArgs& g, uint8_t* smem, uint64_t* full,
                                                uint64_t* empty, int lane) {
    int k = 0;                                        // fills issued
    bool ok = true;
    const int G = g.grab;
    const unsigned long long nitems = (unsigned long long)(g.n_items >= 0 ? g.n_items : *g.n_items_dev);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(g.queue, (unsigned long long)G);
    base = __shfl_sync(0xffffffffu, base, 0);
    TileDesc d{};
    if (lane < G && base + lane < nitems) d = g.desc[base + lane];
    while (ok && base < nitems) {
        unsigned long long nbase = 0;                 // prefetch the next grab
        if (lane == 0) nbase = atomicAdd(g.queue, (unsigned long long)G);
        nbase = __shfl_sync(0xffffffffu, nbase, 0);
        TileDesc nd{};
        if (lane < G && nbase + lane < nitems) nd = g.desc[nbase + lane];
        const int avail = (int)min((unsigned long long)G, nitems - base);
        for (int q = 0; q < avail && ok;) {
            const int64_t a0 = __shfl_sync(0xffffffffu, d.a0, q);
            const int64_t b0 = __shfl_sync(0xffffffffu, d.b0, q);
            const int64_t c0 = __shfl_sync(0xffffffffu, d.c0, q);
            int nA = __shfl_sync(0xffffffffu, d.nA, q);
            int nB = __shfl_sync(0xffffffffu, d.nB, q);
            ++q;
            for (; q < avail; ++q) {                  // pack the following records while they fit
                const int xA = __shfl_sync(0xffffffffu, d.nA, q);
                const int xB = __shfl_sync(0xffffffffu, d.nB, q);
                const int xf = __shfl_sync(0xffffffffu, d.first, q);
                if (xf || nA + nB + xA + xB > g.cap) break;
                nA += xA;
                nB += xB;
            }
            ok = stage_tile<K, V, LOG_T, S_IN, SPLIT>(g, smem, full, empty, lane, k, a0, b0, c0, nA, nB);
        }
        base = nbase;
        d = nd;
    }
    if (ok) stage_end<S_IN, NG>(g, smem, full, empty, lane, k);
}

// Fused single merge, Steps 3-4 selection done by each CTA for itself: the
// subproblems of A-side PEs ca + lane and B-side PEs cb + lane (lanes whose
// PE is below `end` and whose block is not empty), with their indices on the
// merge-path chain, from the cross ranks this launch wrote (read through L2).
// The cross ranks of a PE and of the next one are loaded together in one
// round; the one further rank the split-point form may need (ybar of the
// first B block at or after xbar_i, xbar of the first A block at or after
// ybar_j) usually lies in the other side's window, so it comes from a lane
// of the warp, and from L2 only when it does not.  Lanes without a record
// get chain = INT64_MAX.
struct FusedRec { int64_t a0, b0, chain; int32_t nA, nB; };

__device__ __forceinline__ void fused_records(const EngineArgs& g, int64_t ca, int64_t cb, int64_t end, int lane,
                                              FusedRec& ra, FusedRec& rb) {
    const int64_t n = g.lenA, m = g.lenB, p = g.fp;
    const long long* fx = reinterpret_cast<const long long*>(g.fx);
    const long long* fy = reinterpret_cast<const long long*>(g.fy);
    const int64_t i = ca + lane, j = cb + lane;
    const Blocks32& bA = g.fbA;
    const Blocks32& bB = g.fbB;
    const bool va = i < end && bA.start(i) < n;
    const bool vb = j < end && bB.start(j) < m;
    // one round: xbar_i, xbar_{i+1}, ybar_j, ybar_{j+1} (indices <= p)
    const int64_t xa = va ? (int64_t)__ldcg(fx + i) : 0, xa1 = va ? (int64_t)__ldcg(fx + i + 1) : 0;
    const int64_t ya = vb ? (int64_t)__ldcg(fy + j) : 0, ya1 = vb ? (int64_t)__ldcg(fy + j + 1) : 0;
    // the further rank of each side, from the other side's window when it is there
    const int64_t jn = va ? bB.first_at_or_after(xa) : cb;
    const int64_t in = vb ? bA.first_at_or_after(ya) : ca;
    const int64_t dj = jn - cb, di = in - ca;
    const int64_t yw = __shfl_sync(0xffffffffu, ya, (int)(dj >= 0 && dj < 32 ? dj : 0));
    const int64_t yw1 = __shfl_sync(0xffffffffu, ya1, 31);
    const int64_t xw = __shfl_sync(0xffffffffu, xa, (int)(di >= 0 && di < 32 ? di : 0));
    const int64_t xw1 = __shfl_sync(0xffffffffu, xa1, 31);
    // the window holds ybar[cb .. cb + 32] of valid lanes only: lane 31's
    // ybar_{j+1} counts when lane 31 is valid, any lane's ybar_j when it is
    const bool yin = dj >= 0 && dj < 32 && cb + dj < end && bB.start(cb + dj) < m;
    const bool yin1 = dj == 32 && cb + 31 < end && bB.start(cb + 31) < m;
    const bool xin = di >= 0 && di < 32 && ca + di < end && bA.start(ca + di) < n;
    const bool xin1 = di == 32 && ca + 31 < end && bA.start(ca + 31) < n;
    ra = FusedRec{0, 0, INT64_MAX, 0, 0};
    rb = FusedRec{0, 0, INT64_MAX, 0, 0};
    if (va) {
        // subproblem_of asks an A-side PE for xbar(i), xbar(i+1) and ybar(jn) only
        auto xq = [&](int64_t k) { return k == i ? xa : xa1; };
        auto yq = [&](int64_t k) {
            return yin ? yw : (yin1 ? yw1 : (int64_t)__ldcg(fy + k));
        };
        int64_t a0, a1, b0, b1;
        subproblem_in<int64_t>(true, i, p, bA, bB, xq, yq, a0, a1, b0, b1);
        ra = FusedRec{a0, b0, i + jn, (int32_t)(a1 - a0), (int32_t)(b1 - b0)};
    }
    if (vb) {
        // and a B-side PE for ybar(j), ybar(j+1) and xbar(in) only
        auto yq = [&](int64_t k) { return k == j ? ya : ya1; };
        auto xq = [&](int64_t k) {
            return xin ? xw : (xin1 ? xw1 : (int64_t)__ldcg(fx + k));
        };
        int64_t a0, a1, b0, b1;
        subproblem_in<int64_t>(false, j, p, bA, bB, xq, yq, a0, a1, b0, b1);
        rb = FusedRec{a0, b0, j + in, (int32_t)(a1 - a0), (int32_t)(b1 - b0)};
    }
}

// Producer of the fused single merge.  CTA c owns the processing elements
// [c p / G, (c+1) p / G) of both sides (G CTAs), computes their subproblems
// itself (no records are published, so no second grid barrier), takes them
// in merge-path order and packs chain-adjacent ones (consecutive chain
// indices: contiguous in A, B and C) into tiles of at most `cap` elements.
// Lanes hold up to 32 records of each side at a time.
template <typename K, typename V, int LOG_T, int S_IN, int SPLIT, int NG = 1>
__device__ __forceinline__ void engine_producer_static(const EngineArgs& g, uint8_t* smem, uint64_t* full,
                                                       uint64_t* empty, int lane) {
    const int64_t p = g.fp, G = gridDim.x, c = blockIdx.x;
    const int64_t i0 = c * p / G, i1 = (c + 1) * p / G;
    int64_t ca = i0, cb = i0;                         // first PE of the batch held in the lanes
    FusedRec ra, rb;
    fused_records(g, ca, cb, i1, lane, ra, rb);
    if (g.trace != nullptr && lane == 0) {            // selection of the first records done
        const uint64_t t = global_timer_ns();
        g.trace[(size_t)kTraceSlots * (blockIdx.x + 1) + 3] = t;
        g.trace[(size_t)kTraceSlots * (blockIdx.x + 1) + 4] = t;
    }
    int qa = 0, qb = 0, k = 0;
    bool ok = true;
    int64_t ta0 = 0, tb0 = 0, tnext = -1;             // the tile being packed
    int tA = 0, tB = 0;
    while (ok) {
        if (qa == 32 || qb == 32) {                   // next window of the exhausted side
            FusedRec na, nb;
            if (qa == 32) { ca += 32; qa = 0; }
            if (qb == 32) { cb += 32; qb = 0; }
            fused_records(g, ca, cb, i1, lane, na, nb);
            if (qa == 0) ra = na;
            if (qb == 0) rb = nb;
        }
        const int64_t cha = __shfl_sync(0xffffffffu, ra.chain, qa);
        const int64_t chb = __shfl_sync(0xffffffffu, rb.chain, qb);
        if (cha == INT64_MAX && chb == INT64_MAX) break;
        const bool takeA = cha < chb;                 // warp-uniform
        const FusedRec& r = takeA ? ra : rb;
        const int q = takeA ? qa : qb;
        const int64_t chain = takeA ? cha : chb;
        const int64_t a0 = __shfl_sync(0xffffffffu, r.a0, q);
        const int64_t b0 = __shfl_sync(0xffffffffu, r.b0, q);
        const int nA = __shfl_sync(0xffffffffu, r.nA, q);
        const int nB = __shfl_sync(0xffffffffu, r.nB, q);
        if (takeA) ++qa; else ++qb;
        if (chain == tnext && tA + tB + nA + nB <= g.cap) {   // extends the tile along the merge path
            tA += nA;
            tB += nB;
            ++tnext;
            continue;
        }
        ok = stage_tile<K, V, LOG_T, S_IN, SPLIT>(g, smem, full, empty, lane, k, ta0, tb0, ta0 + tb0, tA, tB);
        ta0 = a0; tb0 = b0; tA = nA; tB = nB; tnext = chain + 1;
    }
    if (ok) ok = stage_tile<K, V, LOG_T, S_IN, SPLIT>(g, smem, full, empty, lane, k, ta0, tb0, ta0 + tb0, tA, tB);
    if (ok) stage_end<S_IN, NG>(g, smem, full, empty, lane, k);
}

// Prefetch into L2 of this CTA's share (1/parts, 16-byte granules, inside the
// array's own aligned span) of an array of len elements of E bytes.
__device__ __forceinline__ void prefetch_share_l2(const void* base, int64_t len, uint32_t E, int64_t part,
                                                  int64_t parts) {
    if (base == nullptr || len <= 0) return;
    const uint64_t b = reinterpret_cast<uint64_t>(base);
    const uint64_t lo = (b + 15) & ~15ull, hi = (b + (uint64_t)len * E) & ~15ull;
    if (hi <= lo) return;
    const uint64_t per = (((hi - lo) + parts - 1) / parts + 15) & ~15ull;
    const uint64_t s = lo + (uint64_t)part * per;
    if (s >= hi) return;
    const uint64_t e = s + per < hi ? s + per : hi;
    for (uint64_t x = s; x < e; x += (1ull << 30)) {
        const uint32_t sz = (uint32_t)((e - x) < (1ull << 30) ? (e - x) : (1ull << 30));
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(x), "r"(sz) : "memory");
    }
}

// Consumers, paper's rule inside the CTA (output via separate buffers).
template <typename K, typename V, int LOG_T, int S_IN, int S_OUT>
__device__ __forceinline__ void engine_consumers_blocks(const EngineArgs& g, uint8_t* smem, uint64_t* full,
                                                        uint64_t* empty, int tid) {
    constexpr int T = 1 << LOG_T;
    int* xs = reinterpret_cast<int*>(smem + g.lay.split_off);
    int* ys = xs + (T + 1);
    const bool leader = (tid == 0);
    for (int k = 0;; ++k) {
        const int s = k % S_IN;
        const int ob = k % S_OUT;
        uint8_t* st = smem + g.lay.stages_off + (uint32_t)s * g.lay.stage_bytes;
        if (!mbar_wait_bounded(&full[s], (k / S_IN) & 1, g.wait_ns)) {
            if (leader) set_status(g.status, TM_ERR_TIMEOUT);
            break;
        }
        const StageHeader* h = reinterpret_cast<const StageHeader*>(st);
        if (h->end) break;
        const int nA = h->nA, nB = h->nB;
        const int64_t c0 = h->c0;
        const K* kA = reinterpret_cast<const K*>(st + g.lay.keys_off + h->kA);
        const K* kB = reinterpret_cast<const K*>(st + g.lay.keys_off + h->kB);
        const V* vA = reinterpret_cast<const V*>(st + g.lay.vals_off + h->vA);
        const V* vB = reinterpret_cast<const V*>(st + g.lay.vals_off + h->vB);
        const BlockSplit<LOG_T> SA(nA, h->mA1, h->mA0), SB(nB, h->mB1, h->mB0);
        uint8_t* ob_base = smem + g.lay.outs_off + (uint32_t)ob * g.lay.out_bytes;
        const uintptr_t gk = reinterpret_cast<uintptr_t>(g.C) + (uintptr_t)c0 * sizeof(K);
        const uintptr_t gv = reinterpret_cast<uintptr_t>(g.Cv) + (uintptr_t)c0 * sizeof(V);
        K* oK = reinterpret_cast<K*>(ob_base + (gk & 15));
        V* oV = reinterpret_cast<V*>(ob_base + g.lay.out_vals_off + (gv & 15));

        // Steps 1-2 inside the tile
        {
            const int xa = SA.start(tid), yb = SB.start(tid);
            const K kx = kA[xa < nA ? xa : 0];
            const K ky = kB[yb < nB ? yb : 0];
            int rl, rh;
            rank_pair_smem(kB, nB, kx, rl, kA, nA, ky, rh);
            xs[tid] = (xa < nA) ? rl : nB;
            ys[tid] = (yb < nB) ? rh : nA;
            if (tid == 0) { xs[T] = nB; ys[T] = nA; }
        }
        if (leader && k >= S_OUT) bulk_wait_read<S_OUT - 1>();   // output buffer ob is free again
        consumer_sync(T);
        // Steps 3-4 inside the tile: A-side item tid, then B-side item tid
        {
            const int xa = SA.start(tid), xa1 = SA.start(tid + 1);
            const int xb = xs[tid], xb1 = xs[tid + 1];
            const int jn = SB.first_at_or_after(xb);
            const int yjn = SB.start(jn);
            int a1, b1;
            if (jn < T && yjn < xb1) { a1 = ys[jn]; b1 = yjn; } else { a1 = xa1; b1 = xb1; }
            merge_run(kA, vA, xa, a1, kB, vB, xb, b1, oK, oV);
        }
        {
            const int yb = SB.start(tid), yb1s = SB.start(tid + 1);
            const int ya = ys[tid], ya1 = ys[tid + 1];
            const int in = SA.first_at_or_after(ya);
            const int xin = SA.start(in);
            int a1, b1;
            if (in < T && xin < ya1) { b1 = xs[in]; a1 = xin; } else { b1 = yb1s; a1 = ya1; }
            merge_run(kA, vA, ya, a1, kB, vB, yb, b1, oK, oV);
        }
        fence_proxy_async_smem();
        consumer_sync(T);
        if (leader) mbar_arrive_expect_tx(&empty[s], 0);         // input stage s may be refilled
        const int L = nA + nB;
        store_out<K>(ob_base, g.C, c0, L, tid, T, leader);
        store_out<V>(ob_base + g.lay.out_vals_off, g.Cv, c0, L, tid, T, leader);
        if (leader) bulk_commit();
    }
    if (leader) bulk_wait_read<0>();
}

// Consumers, equal output runs of VT elements per thread, results written
// back into the consumed stage.  The stage is released one tile later, once
// its bulk store has read it.  NG groups of T threads take the fills in
// turn (group j: fills j, j + NG, ...), each with its own named barrier, so
// that NG tiles of a CTA are merged at once; with S_IN = 2 NG every group
// owns its own pair of stages.
template <typename K, typename V, int LOG_T, int S_IN, int VT, bool VALS, int NG = 1>
__device__ __forceinline__ void engine_consumers_diagonal(const EngineArgs& g, uint8_t* smem, uint64_t* full,
                                                          uint64_t* empty, int ctid) {
    constexpr int T = 1 << LOG_T;
    static_assert(NG == 1 || S_IN == 2 * NG, "a group needs two stages of its own");
    const int grp = ctid >> LOG_T, tid = ctid & (T - 1), bar = 1 + grp;
    const bool leader = (tid == 0);
    int pending = -1;                                  // stage whose store is still reading it
    int k = grp;
    for (;; k += NG) {
        const int s = k % S_IN;
        uint8_t* st = smem + g.lay.stages_off + (uint32_t)s * g.lay.stage_bytes;
        if (!mbar_wait_bounded(&full[s], (k / S_IN) & 1, g.wait_ns)) {
            if (leader) set_status(g.status, TM_ERR_TIMEOUT);
            break;
        }
        if (k == 0 && leader && g.trace != nullptr)       // group 0's first tile
            g.trace[(size_t)kTraceSlots * (blockIdx.x + 1) + 6] = global_timer_ns();
        const StageHeader* h = reinterpret_cast<const StageHeader*>(st);
        if (h->end) break;
        const int nA = h->nA, nB = h->nB;
        const int64_t c0 = h->c0;
        const K* kA = reinterpret_cast<const K*>(st + g.lay.keys_off + h->kA);
        const K* kB = reinterpret_cast<const K*>(st + g.lay.keys_off + h->kB);
        const V* vA = reinterpret_cast<const V*>(st + g.lay.vals_off + h->vA);
        const V* vB = reinterpret_cast<const V*>(st + g.lay.vals_off + h->vB);
        const int L = nA + nB;
        const int d0 = tid * VT;
        const int cnt = max(0, min(VT, L - d0));
        constexpr bool vals = VALS;                    // false: keys-only merge
        K rk[VT];
        V rv[VT];
        if (cnt > 0 && (nA == 0 || nB == 0)) {         // one side empty (Step 3 case (a), its mirror): a copy
            const K* ks = nB == 0 ? kA : kB;
            const V* vs = nB == 0 ? vA : vB;
#pragma unroll
            for (int q = 0; q < VT; ++q) {
                if (q < cnt) {
                    rk[q] = ks[d0 + q];
                    if constexpr (vals) rv[q] = vs[d0 + q];
                }
            }
        } else if (cnt > 0) {
            int i = corank_smem(kA, nA, kB, nB, d0);
            int j = d0 - i;
            K ka = kA[i], kb = kB[j];
#pragma unroll
            for (int q = 0; q < VT; ++q) {
                if (q < cnt) {
                    const bool takeB = (j < nB) && ((i >= nA) || (kb < ka));
                    const int idx = takeB ? j : i;
                    const K* ks = takeB ? kB : kA;
                    const V* vs = takeB ? vB : vA;
                    rk[q] = takeB ? kb : ka;
                    if constexpr (vals) rv[q] = vs[idx];
                    const K nxt = ks[idx + 1];
                    if (takeB) { kb = nxt; ++j; } else { ka = nxt; ++i; }
                }
            }
        }
        consumer_sync(T, bar);                              // all reads of the stage's input done
        const uintptr_t gk = reinterpret_cast<uintptr_t>(g.C) + (uintptr_t)c0 * sizeof(K);
        const uintptr_t gv = reinterpret_cast<uintptr_t>(g.Cv) + (uintptr_t)c0 * sizeof(V);
        uint8_t* bk = st + g.lay.keys_off;
        uint8_t* bv = st + g.lay.vals_off;
        K* oK = reinterpret_cast<K*>(bk + (gk & 15));
        V* oV = reinterpret_cast<V*>(bv + (gv & 15));
#pragma unroll
        for (int q = 0; q < VT; ++q) {
            if (q < cnt) {
                oK[d0 + q] = rk[q];
                if constexpr (vals) oV[d0 + q] = rv[q];
            }
        }
        fence_proxy_async_smem();
        consumer_sync(T, bar);
        store_out<K>(bk, g.C, c0, L, tid, T, leader);
        if constexpr (vals) store_out<V>(bv, g.Cv, c0, L, tid, T, leader);
        if (leader) {
            bulk_commit();
            if (pending >= 0) {                         // previous tile's store has read its stage
                bulk_wait_read<1>();
                mbar_arrive_expect_tx(&empty[pending], 0);
            }
            pending = s;
        }
    }
    if (leader) bulk_wait_read<0>();
    if (leader && grp == 0 && g.trace != nullptr)        // fills taken by the CTA (the end markers excluded)
        g.trace[(size_t)kTraceSlots * (blockIdx.x + 1) + 7] = (uint64_t)(k - grp);
}

template <typename K, typename V, int LOG_T, int S_IN, int S_OUT, int SPLIT, int VT, bool FUSED = false, int NG = 1>
__global__ void __launch_bounds__((1 << LOG_T) * NG + 32)
merge_engine_kernel(const EngineArgs g) {
    constexpr int T = (1 << LOG_T) * NG;              // consumer threads (NG groups), then the producer warp
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + g.lay.bars_off);
    uint64_t* empty = full + S_IN;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < S_IN; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    trace_stamp(g, 0);
    if constexpr (FUSED) {                            // the inputs of the whole merge into L2, in G shares
        if (tid == T) {
            const int64_t c = blockIdx.x, G = gridDim.x;
            const uint32_t vb = g.Cv ? (uint32_t)sizeof(V) : 0u;
            prefetch_share_l2(g.A, g.lenA, sizeof(K), c, G);
            prefetch_share_l2(g.B, g.lenB, sizeof(K), c, G);
            if (vb) {
                prefetch_share_l2(g.Av, g.lenA, vb, c, G);
                prefetch_share_l2(g.Bv, g.lenB, vb, c, G);
            }
        }
    }
    __syncthreads();
    if constexpr (FUSED) {                            // Steps 1-2 and the single synchronisation
        fused_cross_ranks<K>(g);
        trace_stamp(g, 1);
        if (!grid_barrier(g.gbar, 1, g.wait_ns, g.status)) return;
        trace_stamp(g, 2);
    }
    if (tid >= T) {                                   // Steps 3-4: selection by the producer, then merges
        if constexpr (FUSED) engine_producer_static<K, V, LOG_T, S_IN, SPLIT, NG>(g, smem, full, empty, tid - T);
        else                 engine_producer<K, V, LOG_T, S_IN, SPLIT, NG>(g, smem, full, empty, tid - T);
        return;
    }
    if constexpr (SPLIT == kSplitDiagonal) {           // payloads or keys only: one branch per launch
        if (g.Cv != nullptr) engine_consumers_diagonal<K, V, LOG_T, S_IN, VT, true, NG>(g, smem, full, empty, tid);
        else                 engine_consumers_diagonal<K, V, LOG_T, S_IN, VT, false, NG>(g, smem, full, empty, tid);
    } else {
        static_assert(SPLIT == kSplitDiagonal || NG == 1, "one consumer group with the paper's in-CTA rule");
        engine_consumers_blocks<K, V, LOG_T, S_IN, S_OUT>(g, smem, full, empty, tid);
    }
    if constexpr (NG > 1) {
        if (g.trace != nullptr) consumer_sync(T, 15);  // the end stamp after every group's last tile
    }
    trace_stamp(g, 5);
}

}  // namespace pmerge
