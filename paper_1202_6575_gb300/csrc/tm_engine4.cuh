// Persistent tile engine for two merge rounds fused into one pass (the
// stable merge sort of Section 3): each tile holds pieces of four sorted
// runs R0..R3 and the CTA merges them as merge(merge(R0, R1), merge(R2, R3))
// -- the two pairwise merges of one round, then the merge of their results
// of the next round -- with the intermediate sequences in shared memory, so
// that HBM sees each element once per two rounds.
//
// The records come from the paper's method applied to the outer merge of
// X = merge(R0, R1) and Y = merge(R2, R3) (p blocks of X and of Y, cross
// ranks of the block starts, the five cases); every chain point carries the
// offsets it splits the four runs at, so a record is four contiguous
// ranges.  Equal keys keep the order R0, R1, R2, R3 and, inside a run, the
// input order: stable.
//
// CTA = 1 producer warp (lanes 0..7 stage the four key pieces and the four
// payload pieces with cp.async.bulk on the stage's mbarrier) + T consumer
// threads (equal output runs of VT elements in each of the two levels).
#pragma once

#include "tm_engine.cuh"

namespace pmerge {

// One subproblem of a fused pair of rounds: run k contributes
// src[s[k], s[k] + l[k]); the output starts at c0.  Consecutive records of
// one group of four runs are adjacent (all four ranges contiguous).
struct __align__(16) Tile4Desc {
    int64_t s[4];
    int64_t c0;
    int32_t l[4];
    int32_t first, pad0;
};
static_assert(sizeof(Tile4Desc) == 64, "descriptor layout");

struct Stage4Header {
    int64_t c0;
    int32_t l[4];
    uint32_t k[4], v[4];         // byte offsets of element 0 of each piece within its region
    int32_t end;                 // 1: no more tiles
};

struct Engine4Layout {
    uint32_t stage_bytes, keys_off, vals_off;   // within a stage
    uint32_t stages_off;
    uint32_t scratch_k, scratch_v;              // the intermediate X | Y
    uint32_t total;
};

__host__ __device__ inline Engine4Layout make_engine4_layout(int cap, int ksize, int vsize, int s_in) {
    Engine4Layout L;
    // four pieces, each starting on a 16-byte boundary, one element of
    // slack read past a piece's end: 4 * 32 bytes beyond the elements
    const uint32_t kreg = ru128((uint32_t)cap * ksize + 4 * 32 + 96);
    const uint32_t vreg = vsize ? ru128((uint32_t)cap * vsize + 4 * 32 + 96) : 0u;
    L.keys_off = 128;
    L.vals_off = 128 + kreg;
    L.stage_bytes = 128 + kreg + vreg;
    L.stages_off = 128;                                 // after 2 * s_in mbarriers
    uint32_t o = L.stages_off + (uint32_t)s_in * L.stage_bytes;
    L.scratch_k = o;
    o += ru128((uint32_t)cap * ksize + 64);
    L.scratch_v = o;
    o += vsize ? ru128((uint32_t)cap * vsize + 64) : 0u;
    L.total = o;
    return L;
}

struct Engine4Args {
    const Tile4Desc* desc;
    int64_t n_items;
    unsigned long long* queue;     // work-queue counter, zero at launch
    int32_t* status;
    const void* src; const void* srcv; int64_t len;    // the runs (one array) and their payloads
    void* C; void* Cv;                                  // NULL Cv: keys only
    int cap;                       // max sum of l[] of a tile
    int grab;
    uint64_t wait_ns;
    Engine4Layout lay;
};

// Producer warp: pulls records from the work queue, packs consecutive ones
// of the same group of runs while they fit `cap`, and stages the eight
// pieces of each tile (lane 2k: keys of run k, lane 2k+1: its payloads).
template <typename K, typename V, int S_IN>
__device__ __forceinline__ void engine4_producer(const Engine4Args& g, uint8_t* smem, uint64_t* full,
                                                 uint64_t* empty, int lane) {
    int k = 0;
    bool ok = true;
    const int G = g.grab;
    const unsigned long long nitems = (unsigned long long)g.n_items;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(g.queue, (unsigned long long)G);
    base = __shfl_sync(0xffffffffu, base, 0);
    while (ok && base < nitems) {
        const int avail = (int)min((unsigned long long)G, nitems - base);
        Tile4Desc d{};
        if (lane < avail) d = g.desc[base + lane];
        unsigned long long nbase = 0;                 // the next grab, in flight meanwhile
        if (lane == 0) nbase = atomicAdd(g.queue, (unsigned long long)G);
        for (int q = 0; q < avail && ok;) {
            int64_t s[4];
            int l[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                s[r] = __shfl_sync(0xffffffffu, d.s[r], q);
                l[r] = __shfl_sync(0xffffffffu, d.l[r], q);
            }
            const int64_t c0 = __shfl_sync(0xffffffffu, d.c0, q);
            ++q;
            for (; q < avail; ++q) {                  // pack the following records while they fit
                int x[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) x[r] = __shfl_sync(0xffffffffu, d.l[r], q);
                const int xf = __shfl_sync(0xffffffffu, d.first, q);
                if (xf || l[0] + l[1] + l[2] + l[3] + x[0] + x[1] + x[2] + x[3] > g.cap) break;
#pragma unroll
                for (int r = 0; r < 4; ++r) l[r] += x[r];
            }
            const int L = l[0] + l[1] + l[2] + l[3];
            if (L == 0) continue;
            bool inside = true;                       // every range inside the array
#pragma unroll
            for (int r = 0; r < 4; ++r) inside = inside && l[r] >= 0 && s[r] >= 0 && s[r] + l[r] <= g.len;
            if (!inside || L > g.cap) {
                if (lane == 0) set_status(g.status, TM_ERR_BOUNDS);
                continue;
            }
            const int st_i = k % S_IN;
            int free_ok = 1;
            if (lane == 0 && k >= S_IN)
                free_ok = mbar_wait_bounded(&empty[st_i], ((k / S_IN) & 1) ^ 1, g.wait_ns) ? 1 : 0;
            free_ok = __shfl_sync(0xffffffffu, free_ok, 0);
            if (!free_ok) {
                if (lane == 0) set_status(g.status, TM_ERR_TIMEOUT);
                ok = false;
                break;
            }
            uint8_t* st = smem + g.lay.stages_off + (uint32_t)st_i * g.lay.stage_bytes;
            const int piece = (lane >> 1) & 3;
            const bool isV = (lane & 1) != 0;
            const uint32_t E = isV ? (uint32_t)sizeof(V) : (uint32_t)sizeof(K);
            const void* pbase = isV ? g.srcv : g.src;
            // every lane walks the pieces of its region in order: piece r + 1
            // starts on the 16-byte boundary after piece r's bytes plus 16
            uint32_t dst_off = 0;
            const uintptr_t b = reinterpret_cast<uintptr_t>(pbase);
            for (int r = 0; r < piece; ++r)
                dst_off = (dst_off + (uint32_t)((b + (uintptr_t)s[r] * E) & 15) + (uint32_t)l[r] * E + 31u) & ~15u;
            const int64_t pcnt = (isV && g.Cv == nullptr) ? 0 : (int64_t)(piece == 0 ? l[0] : piece == 1 ? l[1]
                                                                        : piece == 2 ? l[2] : l[3]);
            const int64_t plo = piece == 0 ? s[0] : piece == 1 ? s[1] : piece == 2 ? s[2] : s[3];
            uint8_t* region = st + (isV ? g.lay.vals_off : g.lay.keys_off);
            uint32_t tx = 0, off = 0;
            if (lane < 8) off = stage_piece(region, dst_off, pbase, g.len, plo, pcnt, E, &full[st_i], tx, 0);
#pragma unroll
            for (int sh = 1; sh < 8; sh <<= 1) tx += __shfl_xor_sync(0xffffffffu, tx, sh);
            uint32_t offs[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) offs[r] = __shfl_sync(0xffffffffu, off, r);
            __syncwarp();                              // plain edge loads before the arrive
            if (lane == 0) {
                Stage4Header* h = reinterpret_cast<Stage4Header*>(st);
                h->c0 = c0;
#pragma unroll
                for (int r = 0; r < 4; ++r) { h->l[r] = l[r]; h->k[r] = offs[2 * r]; h->v[r] = offs[2 * r + 1]; }
                h->end = 0;
                mbar_arrive_expect_tx(&full[st_i], tx);
            }
            __syncwarp();
            uint32_t unused = 0;
            if (lane < 8) stage_piece(region, dst_off, pbase, g.len, plo, pcnt, E, &full[st_i], unused, 1);
            ++k;
        }
        base = __shfl_sync(0xffffffffu, nbase, 0);
    }
    if (lane == 0 && ok) {                            // end marker for the consumers
        const int st_i = k % S_IN;
        if (k >= S_IN && !mbar_wait_bounded(&empty[st_i], ((k / S_IN) & 1) ^ 1, g.wait_ns)) {
            set_status(g.status, TM_ERR_TIMEOUT);
        } else {
            Stage4Header* h = reinterpret_cast<Stage4Header*>(smem + g.lay.stages_off +
                                                              (uint32_t)st_i * g.lay.stage_bytes);
            h->end = 1;
            mbar_arrive_expect_tx(&full[st_i], 0);
        }
    }
}

// Outputs [e0, e0 + cnt) of the stable merge of P (nP) and Q (nQ) in
// shared memory (P first on equal keys) into o[e0..]: the co-rank of e0 by
// the position formulas of Section 2, then a serial merge.
template <typename K, typename V, bool VALS>
__device__ __forceinline__ void merge_part(const K* kP, const V* vP, int nP, const K* kQ, const V* vQ, int nQ,
                                           int e0, int cnt, K* oK, V* oV) {
    if (cnt <= 0) return;
    int i = corank_smem(kP, nP, kQ, nQ, e0);
    int j = e0 - i;
    K kp = kP[i], kq = kQ[j];
    for (int q = 0; q < cnt; ++q) {
        const bool takeQ = (j < nQ) && ((i >= nP) || (kq < kp));
        const int idx = takeQ ? j : i;
        const K* ks = takeQ ? kQ : kP;
        oK[e0 + q] = takeQ ? kq : kp;
        if constexpr (VALS) oV[e0 + q] = (takeQ ? vQ : vP)[idx];
        const K nxt = ks[idx + 1];
        if (takeQ) { kq = nxt; ++j; } else { kp = nxt; ++i; }
    }
}

// Consumers: level 1 writes X = merge(R0, R1) and Y = merge(R2, R3) side by
// side into the scratch (thread t: outputs [t VT, t VT + VT) of X | Y, which
// may straddle the two); level 2 merges X and Y (X first on equal keys)
// into registers, VT outputs per thread, writes them back into the consumed
// stage and stores them from there, as the two-run engine does.
template <typename K, typename V, int LOG_T, int S_IN, int VT, bool VALS>
__device__ __forceinline__ void engine4_consumers(const Engine4Args& g, uint8_t* smem, uint64_t* full,
                                                  uint64_t* empty, int tid) {
    constexpr int T = 1 << LOG_T;
    const bool leader = (tid == 0);
    K* xk = reinterpret_cast<K*>(smem + g.lay.scratch_k);
    V* xv = reinterpret_cast<V*>(smem + g.lay.scratch_v);
    int pending = -1;
    for (int k = 0;; ++k) {
        const int s = k % S_IN;
        uint8_t* st = smem + g.lay.stages_off + (uint32_t)s * g.lay.stage_bytes;
        if (!mbar_wait_bounded(&full[s], (k / S_IN) & 1, g.wait_ns)) {
            if (leader) set_status(g.status, TM_ERR_TIMEOUT);
            break;
        }
        const Stage4Header* h = reinterpret_cast<const Stage4Header*>(st);
        if (h->end) break;
        const int l0 = h->l[0], l1 = h->l[1], l2 = h->l[2], l3 = h->l[3];
        const int64_t c0 = h->c0;
        const int nX = l0 + l1, L = nX + l2 + l3;
        const K* k0 = reinterpret_cast<const K*>(st + g.lay.keys_off + h->k[0]);
        const K* k1 = reinterpret_cast<const K*>(st + g.lay.keys_off + h->k[1]);
        const K* k2 = reinterpret_cast<const K*>(st + g.lay.keys_off + h->k[2]);
        const K* k3 = reinterpret_cast<const K*>(st + g.lay.keys_off + h->k[3]);
        const V* v0 = reinterpret_cast<const V*>(st + g.lay.vals_off + h->v[0]);
        const V* v1 = reinterpret_cast<const V*>(st + g.lay.vals_off + h->v[1]);
        const V* v2 = reinterpret_cast<const V*>(st + g.lay.vals_off + h->v[2]);
        const V* v3 = reinterpret_cast<const V*>(st + g.lay.vals_off + h->v[3]);
        const int d0 = tid * VT;
        const int d1 = min(d0 + VT, L);
        // level 1 (the scratch is free: the previous tile's level 2 read it
        // before the barrier that ended its write-back)
        if (d0 < nX) merge_part<K, V, VALS>(k0, v0, l0, k1, v1, l1, d0, min(d1, nX) - d0, xk, xv);
        if (d1 > nX) {
            const int e0 = max(d0, nX) - nX;
            merge_part<K, V, VALS>(k2, v2, l2, k3, v3, l3, e0, d1 - max(d0, nX), xk + nX, xv + nX);
        }
        consumer_sync(T);
        // level 2: X = scratch[0, nX), Y = scratch[nX, L)
        const int cnt = max(0, d1 - d0);
        K rk[VT];
        V rv[VT];
        if (cnt > 0) {
            const K* kX = xk; const K* kY = xk + nX;
            const V* vX = xv; const V* vY = xv + nX;
            const int nY = L - nX;
            int i = corank_smem(kX, nX, kY, nY, d0);
            int j = d0 - i;
            K ka = kX[i], kb = kY[j];
#pragma unroll
            for (int q = 0; q < VT; ++q) {
                if (q < cnt) {
                    const bool takeB = (j < nY) && ((i >= nX) || (kb < ka));
                    const int idx = takeB ? j : i;
                    const K* ks = takeB ? kY : kX;
                    rk[q] = takeB ? kb : ka;
                    if constexpr (VALS) rv[q] = (takeB ? vY : vX)[idx];
                    const K nxt = ks[idx + 1];
                    if (takeB) { kb = nxt; ++j; } else { ka = nxt; ++i; }
                }
            }
        }
        // the stage's inputs were last read in level 1, before the barrier
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
                if constexpr (VALS) oV[d0 + q] = rv[q];
            }
        }
        fence_proxy_async_smem();
        consumer_sync(T);                              // write-back done; scratch reads done
        store_out<K>(bk, g.C, c0, L, tid, T, leader);
        if constexpr (VALS) store_out<V>(bv, g.Cv, c0, L, tid, T, leader);
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
}

template <typename K, typename V, int LOG_T, int S_IN, int VT>
__global__ void __launch_bounds__((1 << LOG_T) + 32)
merge4_engine_kernel(const Engine4Args g) {
    constexpr int T = 1 << LOG_T;
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + S_IN;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < S_IN; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    if (tid >= T) {
        engine4_producer<K, V, S_IN>(g, smem, full, empty, tid - T);
        return;
    }
    if (g.Cv != nullptr) engine4_consumers<K, V, LOG_T, S_IN, VT, true>(g, smem, full, empty, tid);
    else                 engine4_consumers<K, V, LOG_T, S_IN, VT, false>(g, smem, full, empty, tid);
}

}  // namespace pmerge
