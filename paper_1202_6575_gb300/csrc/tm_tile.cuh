// Staged tile merge: one CTA merges one subproblem (an A range and a B range
// that the cross ranks delimit) held in shared memory.
//
// Staging: each of the four input ranges (A keys, A payloads, B keys,
// B payloads) is fetched with one bulk copy (cp.async.bulk, the TMA engine)
// of its 16-byte-aligned window; elements outside the array's own aligned
// span (only at the very start or end of an array) are fetched with plain
// loads.  Re-split: the CTA applies the paper's rule again, with its T
// threads as the processing elements: T blocks per piece, rank_low of each
// A-block start in the B piece, rank_high of each B-block start in the A
// piece (binary search in shared memory), then the 2T sub-subproblems of the
// split-point form, two per thread, each merged by a short serial stable
// merge.  Output: the merged tile is written to shared memory at the
// misalignment of its global destination and stored with bulk copies
// (16-byte aligned middle) plus plain stores for the ragged ends.
#pragma once

#include "tm_common.cuh"

namespace pmerge {

// Shared-memory layout of one tile stage.  capA/capB: maximum piece lengths.
struct TileLayout {
    uint32_t off_split;   // int32 xs[T+1], ys[T+1]
    uint32_t off_kA, off_vA, off_kB, off_vB, off_kC, off_vC;
    uint32_t bytes;       // total
};

__host__ __device__ inline uint32_t round_up_u32(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline TileLayout make_tile_layout(int capA, int capB, int ksize, int threads) {
    TileLayout L;
    uint32_t o = 128;                                  // mbarrier + header
    L.off_split = o; o = round_up_u32(o + 8u * (threads + 1), 128);
    L.off_kA = o; o = round_up_u32(o + (uint32_t)capA * ksize + 32, 128);
    L.off_vA = o; o = round_up_u32(o + (uint32_t)capA * 4 + 32, 128);
    L.off_kB = o; o = round_up_u32(o + (uint32_t)capB * ksize + 32, 128);
    L.off_vB = o; o = round_up_u32(o + (uint32_t)capB * 4 + 32, 128);
    uint32_t capC = (uint32_t)capA + (uint32_t)capB;
    L.off_kC = o; o = round_up_u32(o + capC * ksize + 16, 128);
    L.off_vC = o; o = round_up_u32(o + capC * 4 + 16, 128);
    L.bytes = o;
    return L;
}

// Geometry of staging elements [lo, hi) of an array (base, len, element size E)
// into a shared region.  The region holds the 16-byte window that starts at
// round_down(&X[lo], 16); X[lo] sits at element offset `head` of the region.
// [t0, t1) is the part a bulk copy fetches (aligned, inside the array's own
// aligned span); the rest of [lo, hi) is fetched with plain loads.
struct StageWin {
    uintptr_t g0, g1, w0, t0, t1;
    uint32_t head;
    __device__ __forceinline__ uint32_t bulk_bytes() const { return t1 > t0 ? (uint32_t)(t1 - t0) : 0u; }
};

__device__ __forceinline__ StageWin stage_window(const void* base, int64_t len, int64_t lo, int64_t hi, int E) {
    StageWin w;
    uintptr_t b = reinterpret_cast<uintptr_t>(base);
    w.g0 = b + (uintptr_t)(lo * E);
    w.g1 = b + (uintptr_t)(hi * E);
    w.w0 = w.g0 & ~(uintptr_t)15;
    uintptr_t lim0 = (b + 15) & ~(uintptr_t)15;
    uintptr_t lim1 = (b + (uintptr_t)(len * E)) & ~(uintptr_t)15;
    uintptr_t r1 = (w.g1 + 15) & ~(uintptr_t)15;
    w.t0 = w.w0 > lim0 ? w.w0 : lim0;
    w.t1 = r1 < lim1 ? r1 : lim1;
    w.head = (uint32_t)((w.g0 - w.w0) / E);
    return w;
}

__device__ __forceinline__ void stage_issue(uint8_t* region, const StageWin& w, uint64_t* bar) {
    if (w.t1 > w.t0)
        bulk_g2s(region + (w.t0 - w.w0), reinterpret_cast<const void*>(w.t0), (uint32_t)(w.t1 - w.t0), bar);
}

// Plain loads of the elements of [g0, g1) the bulk copy does not cover.
template <typename T>
__device__ __forceinline__ void stage_edges(uint8_t* region, const StageWin& w, int tid, int nthreads) {
    const uintptr_t E = sizeof(T);
    uintptr_t c0 = w.t0, c1 = w.t1;
    if (c1 <= c0) { c0 = w.g1; c1 = w.g1; }           // nothing bulk-copied: everything plain
    // head part [g0, min(c0, g1)), tail part [max(c1, g0), g1)
    uintptr_t h1 = c0 < w.g1 ? c0 : w.g1;
    int64_t nh = h1 > w.g0 ? (int64_t)((h1 - w.g0) / E) : 0;
    uintptr_t s0 = c1 > w.g0 ? c1 : w.g0;
    int64_t nt = w.g1 > s0 ? (int64_t)((w.g1 - s0) / E) : 0;
    T* dst = reinterpret_cast<T*>(region) + w.head;
    const T* src = reinterpret_cast<const T*>(w.g0);
    for (int64_t e = tid; e < nh; e += nthreads) dst[e] = src[e];
    int64_t tail0 = (int64_t)((s0 - w.g0) / E);
    for (int64_t e = tid; e < nt; e += nthreads) dst[tail0 + e] = src[tail0 + e];
}

// Serial stable merge of sA[ia0..ia1) and sB[ib0..ib1) into sC from ia0 + ib0.
// B is taken only when its key is strictly smaller: equal keys keep A first.
// Reads one element past a range end, which stays inside the padded region.
template <typename K>
__device__ __forceinline__ void merge_serial(const K* sAk, const uint32_t* sAv, int ia0, int ia1,
                                             const K* sBk, const uint32_t* sBv, int ib0, int ib1,
                                             K* sCk, uint32_t* sCv) {
    int i = ia0, j = ib0, o = ia0 + ib0;
    const int oend = ia1 + ib1;
    K ka = sAk[i];
    K kb = sBk[j];
    while (o < oend) {
        const bool takeB = (j < ib1) && ((i >= ia1) || (kb < ka));
        const K* ks = takeB ? sBk : sAk;
        const uint32_t* vs = takeB ? sBv : sAv;
        const int idx = takeB ? j : i;
        sCk[o] = takeB ? kb : ka;
        sCv[o] = vs[idx];
        const K nxt = ks[idx + 1];
        if (takeB) { kb = nxt; ++j; } else { ka = nxt; ++i; }
        ++o;
    }
}

// Pointers to element 0 of each staged piece and of the output tile.
template <typename K>
struct TileView {
    K* kA; uint32_t* vA; K* kB; uint32_t* vB; K* kC; uint32_t* vC;
    int* xs; int* ys;
};

// In-CTA re-split of a staged subproblem (nA, nB elements) among the CTA's
// T threads and the serial merges into the output tile.  Ends with every
// thread's smem writes fenced for the async proxy and a CTA barrier.
template <typename K>
__device__ __forceinline__ void tile_resplit_and_merge(const TileView<K>& v, int nA, int nB) {
    const int T = blockDim.x, t = threadIdx.x;
    // Steps 1-2 inside the tile: cross ranks of the T block starts per side.
    {
        int xa = block_start(nA, T, t);
        int yb = block_start(nB, T, t);
        v.xs[t] = (xa < nA) ? rank_low_smem(v.kB, nB, v.kA[xa]) : nB;
        v.ys[t] = (yb < nB) ? rank_high_smem(v.kA, nA, v.kB[yb]) : nA;
        if (t == 0) { v.xs[T] = nB; v.ys[T] = nA; }
    }
    __syncthreads();
    // Steps 3-4 inside the tile: A-side item t, then B-side item t.
    auto xbar = [&](int i) { return v.xs[i]; };
    auto ybar = [&](int j) { return v.ys[j]; };
    int a0, a1, b0, b1;
    subproblem_of<int>(true, t, nA, nB, T, xbar, ybar, a0, a1, b0, b1);
    merge_serial(v.kA, v.vA, a0, a1, v.kB, v.vB, b0, b1, v.kC, v.vC);
    subproblem_of<int>(false, t, nA, nB, T, xbar, ybar, a0, a1, b0, b1);
    merge_serial(v.kA, v.vA, a0, a1, v.kB, v.vB, b0, b1, v.kC, v.vC);
    fence_proxy_async_smem();
    __syncthreads();
}

// Output geometry of L elements of size E at global address gc.
struct OutWin {
    uintptr_t g0, g1, m0, m1;   // [m0, m1): 16-byte aligned middle (empty if m1 <= m0)
    uint32_t mis;               // g0 & 15: byte offset of element 0 in the smem region
};

__device__ __forceinline__ OutWin out_window(const void* base, int64_t c0, int64_t L, int E) {
    OutWin w;
    w.g0 = reinterpret_cast<uintptr_t>(base) + (uintptr_t)(c0 * E);
    w.g1 = w.g0 + (uintptr_t)(L * E);
    w.m0 = (w.g0 + 15) & ~(uintptr_t)15;
    w.m1 = w.g1 & ~(uintptr_t)15;
    w.mis = (uint32_t)(w.g0 & 15);
    return w;
}

// Issued by one thread: the bulk store of the aligned middle.
__device__ __forceinline__ void out_issue(const OutWin& w, const uint8_t* region) {
    if (w.m1 > w.m0)
        bulk_s2g(reinterpret_cast<void*>(w.m0), region + w.mis + (w.m0 - w.g0), (uint32_t)(w.m1 - w.m0));
}

// Plain stores of the ragged head and tail (all elements when no middle).
template <typename T>
__device__ __forceinline__ void out_edges(const OutWin& w, const uint8_t* region, int tid, int nthreads) {
    const uintptr_t E = sizeof(T);
    const T* src = reinterpret_cast<const T*>(region + w.mis);
    T* dst = reinterpret_cast<T*>(w.g0);
    int64_t total = (int64_t)((w.g1 - w.g0) / E);
    if (w.m1 <= w.m0) {
        for (int64_t e = tid; e < total; e += nthreads) dst[e] = src[e];
        return;
    }
    int64_t nh = (int64_t)((w.m0 - w.g0) / E);
    int64_t t0 = (int64_t)((w.m1 - w.g0) / E);
    for (int64_t e = tid; e < nh; e += nthreads) dst[e] = src[e];
    for (int64_t e = t0 + tid; e < total; e += nthreads) dst[e] = src[e];
}

}  // namespace pmerge
