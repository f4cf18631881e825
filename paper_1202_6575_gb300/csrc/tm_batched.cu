// Many independent stable merges at once (Section 3: the merge applied in
// parallel to several pairs) and the stable merge sort built from it.
//
// Each pair k gets its own block count p_k and runs the single-merge method:
// cross-rank searches of its block starts (one search kernel over all pairs),
// subproblem selection (one plan kernel over all pairs, records in
// merge-path order per pair), then one launch of the persistent tile engine
// over every pair's records, which pulls them from its device work queue.
// Every grid is sized from host-known bounds and the engine reads the record
// count from device memory, so a whole batched merge is one stream sequence
// with no host synchronisation and can be captured in a CUDA graph.
#include <cstring>
#include <new>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "tm_engine.cuh"
#include "tm_engine4.cuh"
#include "tm_host.h"
#include "tm_runsort.cuh"

namespace pmerge {

// TM_OK, or TM_ERR_CUDA with the pending launch error recorded for
// tm_last_cuda_error.
static tm_status launch_status() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TM_OK : cuda_failed(e);
}

// A set of pairs: either CSR offsets (pair k merges A[a_off[k]..a_off[k+1])
// with B[b_off[k]..b_off[k+1]) into C from a_off[k] + b_off[k]), or
// explicit runs of one array (pair k merges X[a0, a0+n) with the run right
// after it, X[a0+n, a0+n+m), into C from a0; (a0, n, m) = pdesc[3k..3k+2]),
// or uniform runs of one array (pair k merges the sorted runs [2k*run,
// (2k+1)*run) and [(2k+1)*run, (2k+2)*run) of X, clipped to `total`, into C
// from 2k*run).
struct PairSet {
    int64_t num_pairs;
    const int64_t* a_off;
    const int64_t* b_off;
    const int64_t* pdesc;          // explicit mode
    int64_t run, total;            // uniform mode when a_off == pdesc == nullptr
    int64_t p_uniform;             // blocks per pair in uniform mode

    // Per-pair block counts vary (CSR and explicit modes): they are scanned.
    __host__ __device__ __forceinline__ bool scanned() const { return a_off != nullptr || pdesc != nullptr; }

    __device__ __forceinline__ void get(int64_t k, int64_t& a0, int64_t& n, int64_t& b0, int64_t& m,
                                        int64_t& c0) const {
        if (a_off) {
            a0 = a_off[k]; n = a_off[k + 1] - a0;
            b0 = b_off[k]; m = b_off[k + 1] - b0;
            c0 = a0 + b0;
        } else if (pdesc) {
            a0 = pdesc[3 * k]; n = pdesc[3 * k + 1]; m = pdesc[3 * k + 2];
            b0 = a0 + n;
            c0 = a0;
        } else {
            a0 = 2 * k * run;
            n = total - a0 < run ? total - a0 : run;
            b0 = a0 + n;
            m = total - b0 < run ? total - b0 : run;
            if (m < 0) m = 0;
            c0 = a0;
        }
    }
};

// Per-pair block count: enough blocks that one subproblem fits `tile`.
__host__ __device__ __forceinline__ int64_t pair_blocks(int64_t n, int64_t m, int64_t tile) {
    const int64_t len = n + m;
    if (len == 0) return 0;
    const int64_t p = (len + tile - 1) / tile;
    return p < 1 ? 1 : p;
}

__host__ __device__ __forceinline__ int64_t pair_items(int64_t n, int64_t m, int64_t p) {
    return (n < p ? n : p) + (m < p ? m : p);
}

// Bases of pair k (uniform mode: closed form; CSR mode: scanned arrays).
struct PairBases {
    const int64_t* search_base;    // 2 p_k prefix      (CSR)
    const int64_t* rank_base;      // (p_k + 1) prefix  (CSR)
    const int64_t* item_base;      // items prefix      (CSR)
    const int64_t* cta_pair;       // pair of each search/plan CTA's first thread (CSR)
};

// ---------------------------------------------------------------------------
// CSR mode: per-pair counts and their exclusive scans
// ---------------------------------------------------------------------------

// Exclusive scan of three int64 values over a CTA of NT threads (NT a
// multiple of 32, at most 1024): warp shuffles, then the warp totals.
template <int NT>
__device__ __forceinline__ void block_scan3(const int64_t v[3], int64_t ex[3], int64_t tot[3]) {
    __shared__ int64_t wsum[3][NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t in[3] = {v[0], v[1], v[2]};
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int64_t y = __shfl_up_sync(0xffffffffu, in[c], off);
            if (lane >= off) in[c] += y;
        }
    }
    if (lane == 31) { wsum[0][warp] = in[0]; wsum[1][warp] = in[1]; wsum[2][warp] = in[2]; }
    __syncthreads();
    if (warp == 0) {                                   // scan of the warp totals
        int64_t w[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) w[c] = lane < NT / 32 ? wsum[c][lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int64_t y = __shfl_up_sync(0xffffffffu, w[c], off);
                if (lane >= off) w[c] += y;
            }
        }
        if (lane < NT / 32) { wsum[0][lane] = w[0]; wsum[1][lane] = w[1]; wsum[2][lane] = w[2]; }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        ex[c] = in[c] - v[c] + (warp ? wsum[c][warp - 1] : 0);
        tot[c] = wsum[c][NT / 32 - 1];
    }
    __syncthreads();                                   // wsum may be reused by the caller's next scan
}

// Per-pair counts (2 p_k searches, p_k + 1 cross-rank slots, records),
// scanned within the CTA: each pair gets its exclusive prefix within its
// CTA and part[c][blockIdx] the CTA's totals.
__global__ void __launch_bounds__(256)
pair_count_kernel(PairSet ps, int64_t tile, int64_t* __restrict__ cnt_search, int64_t* __restrict__ cnt_rank,
                  int64_t* __restrict__ cnt_item, int64_t* __restrict__ part, int64_t nparts) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t v[3] = {0, 0, 0};
    if (k < ps.num_pairs) {
        int64_t a0, n, b0, m, c0;
        ps.get(k, a0, n, b0, m, c0);
        const int64_t p = pair_blocks(n, m, tile);
        v[0] = 2 * p; v[1] = p + 1; v[2] = pair_items(n, m, p);
    }
    int64_t ex[3], tot[3];
    block_scan3<256>(v, ex, tot);
    if (k < ps.num_pairs) { cnt_search[k] = ex[0]; cnt_rank[k] = ex[1]; cnt_item[k] = ex[2]; }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = tot[0]; part[nparts + blockIdx.x] = tot[1]; part[2 * nparts + blockIdx.x] = tot[2];
    }
}

// Exclusive scan of the CTA totals in place (one CTA, rounds of 1024 with a
// running carry); the grand totals go to base[num] of the three arrays and
// the record total to *n_items.
__global__ void __launch_bounds__(1024)
part_scan_kernel(int64_t* __restrict__ part, int64_t nparts, int64_t num, int64_t* __restrict__ s0,
                 int64_t* __restrict__ s1, int64_t* __restrict__ s2, int64_t* __restrict__ n_items) {
    int64_t carry[3] = {0, 0, 0};
    for (int64_t r = 0; r < nparts; r += 1024) {
        const int64_t i = r + threadIdx.x;
        int64_t v[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] = i < nparts ? part[c * nparts + i] : 0;
        int64_t ex[3], tot[3];
        block_scan3<1024>(v, ex, tot);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (i < nparts) part[c * nparts + i] = carry[c] + ex[c];
            carry[c] += tot[c];
        }
    }
    if (threadIdx.x == 0) {
        s0[num] = carry[0]; s1[num] = carry[1]; s2[num] = carry[2];
        *n_items = carry[2];
    }
}

// Adds each CTA's offset to its pairs' prefixes (the three arrays become
// global exclusive prefixes) and records, for every 256-thread CTA of the
// search and plan kernels whose first thread falls in pair k's searches,
// cta_pair[CTA] = k.
__global__ void __launch_bounds__(256)
part_add_kernel(PairSet ps, int64_t tile, const int64_t* __restrict__ part, int64_t nparts,
                int64_t* __restrict__ s0, int64_t* __restrict__ s1, int64_t* __restrict__ s2,
                int64_t* __restrict__ cta_pair) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ps.num_pairs) return;
    const int64_t sk = s0[k] + part[blockIdx.x];
    s0[k] = sk;
    s1[k] += part[nparts + blockIdx.x];
    s2[k] += part[2 * nparts + blockIdx.x];
    int64_t a0, n, b0, m, c0;
    ps.get(k, a0, n, b0, m, c0);
    const int64_t ek = sk + 2 * pair_blocks(n, m, tile);
    for (int64_t c = (sk + 255) / 256; c * 256 < ek; ++c) cta_pair[c] = k;
}

// Pair owning global search index t: the last k with search_base[k] <= t.
__device__ __forceinline__ int64_t pair_of(const int64_t* base, int64_t num, int64_t t) {
    int64_t lo = 0, len = num;                        // first k with base[k] > t, minus one
    while (len > 0) {
        const int64_t half = len >> 1;
        if (__ldg(base + lo + half + 1) <= t) { lo += half + 1; len -= half + 1; } else { len = half; }
    }
    return lo;
}

// Maps a global (search or plan) thread index to (pair, local index).
__device__ __forceinline__ bool locate(const PairSet& ps, const PairBases& pb, int64_t t, int64_t& k,
                                       int64_t& local, int64_t& p) {
    if (ps.scanned()) {
        if (t >= __ldg(pb.search_base + ps.num_pairs)) return false;
        k = pair_of(pb.search_base, ps.num_pairs, t);
        local = t - __ldg(pb.search_base + k);
        p = (__ldg(pb.search_base + k + 1) - __ldg(pb.search_base + k)) / 2;
    } else {
        p = ps.p_uniform;
        k = div_nonneg<int64_t>(t, 2 * p);
        if (k >= ps.num_pairs) return false;
        local = t - k * 2 * p;
    }
    return true;
}

// The pairs that own one CTA's search (or plan) threads: from the first pair
// of this CTA to the first pair of the next one (cta_pair, written with the
// scan), their search bases staged in shared memory when the range is
// short, so that every thread finds its pair there instead of bisecting the
// whole prefix array in global memory.
constexpr int kPairWin = 512;
struct PairWin { int64_t kf; int cnt; };           // cnt staged bases; 0: not staged

__device__ __forceinline__ PairWin stage_pair_window(const PairSet& ps, const PairBases& pb, int64_t total_threads,
                                                     int64_t* sb) {
    PairWin w{0, 0};
    if (!ps.scanned()) return w;                       // uniform pairs: closed form, the same for every CTA
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x;
    const int64_t all = __ldg(pb.search_base + ps.num_pairs);
    const int64_t tot = all < total_threads ? all : total_threads;
    if (t0 >= tot) return w;                           // uniform over the CTA: no thread of it has work
    const int64_t kf = __ldg(pb.cta_pair + blockIdx.x);
    const int64_t kl = t0 + (int64_t)blockDim.x < tot ? __ldg(pb.cta_pair + blockIdx.x + 1) : ps.num_pairs - 1;
    const int64_t cnt = kl - kf + 2;                   // bases of pairs kf..kl and the end of kl
    if (cnt <= kPairWin) {
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) sb[i] = __ldg(pb.search_base + kf + i);
        w.kf = kf;
        w.cnt = (int)cnt;
    }
    __syncthreads();
    return w;
}

// locate() through the staged window when there is one.
__device__ __forceinline__ bool locate_in(const PairSet& ps, const PairBases& pb, const PairWin& w,
                                          const int64_t* sb, int64_t t, int64_t& k, int64_t& local, int64_t& p) {
    if (ps.scanned() && w.cnt) {
        if (t >= sb[w.cnt - 1]) return false;          // past the last pair's searches
        int lo = 0, len = w.cnt - 1;                    // last i <= cnt-2 with sb[i] <= t
        while (len > 0) {
            const int half = len >> 1;
            if (sb[lo + half + 1] <= t) { lo += half + 1; len -= half + 1; } else { len = half; }
        }
        k = w.kf + lo;
        local = t - sb[lo];
        p = (sb[lo + 1] - sb[lo]) / 2;
        return true;
    }
    return locate(ps, pb, t, k, local, p);
}

__device__ __forceinline__ int64_t rank_base_of(const PairSet& ps, const PairBases& pb, int64_t k) {
    return ps.scanned() ? __ldg(pb.rank_base + k) : k * (ps.p_uniform + 1);
}

__device__ __forceinline__ int64_t item_base_of(const PairSet& ps, const PairBases& pb, int64_t k) {
    return ps.scanned() ? __ldg(pb.item_base + k) : k * 2 * ps.p_uniform;
}

// Steps 1-2 of every pair.
template <typename K>
__global__ void __launch_bounds__(256)
batched_search_kernel(PairSet ps, PairBases pb, const K* __restrict__ A, const K* __restrict__ B,
                      int64_t total_threads, int64_t* __restrict__ xbar, int64_t* __restrict__ ybar) {
    __shared__ int64_t sb[kPairWin];
    const PairWin w = stage_pair_window(ps, pb, total_threads, sb);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total_threads) return;
    int64_t k, local, p;
    if (!locate_in(ps, pb, w, sb, t, k, local, p)) return;
    int64_t a0, n, b0, m, c0;
    ps.get(k, a0, n, b0, m, c0);
    const int64_t rb = rank_base_of(ps, pb, k);
    if (local < p) {
        const int64_t xi = block_start<int64_t>(n, p, local);
        xbar[rb + local] = (xi < n) ? rank_low_global<K, int64_t>(B + b0, m, __ldg(A + a0 + xi)) : m;
        if (local == 0) { xbar[rb + p] = m; ybar[rb + p] = n; }
    } else {
        const int64_t j = local - p;
        const int64_t yj = block_start<int64_t>(m, p, j);
        ybar[rb + j] = (yj < m) ? rank_high_global<K, int64_t>(A + a0, n, __ldg(B + b0 + yj)) : n;
    }
}

// Steps 3-4 selection of every pair: records in merge-path order per pair,
// at global offsets, the pair's first record flagged.
__global__ void __launch_bounds__(256)
batched_plan_kernel(PairSet ps, PairBases pb, int64_t total_threads, const int64_t* __restrict__ xbar,
                    const int64_t* __restrict__ ybar, TileDesc* __restrict__ desc) {
    __shared__ int64_t sb[kPairWin];
    const PairWin w = stage_pair_window(ps, pb, total_threads, sb);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total_threads) return;
    int64_t k, local, p;
    if (!locate_in(ps, pb, w, sb, t, k, local, p)) return;
    int64_t a0g, n, b0g, m, c0g;
    ps.get(k, a0g, n, b0g, m, c0g);
    const bool a_side = local < p;
    const int64_t pe = a_side ? local : local - p;
    if (a_side ? block_start<int64_t>(n, p, pe) >= n : block_start<int64_t>(m, p, pe) >= m) return;
    const int64_t rb = rank_base_of(ps, pb, k);
    int64_t a0, a1, b0, b1, chain;
    constexpr int64_t kSmall = int64_t(1) << 30;       // block arithmetic of such pairs fits int32
    if (n < kSmall && m < kSmall && p < kSmall) {       // 32-bit divisions: every pair of a sort round
        auto xb = [&](int32_t i) { return (int32_t)__ldg(xbar + rb + i); };
        auto yb = [&](int32_t j) { return (int32_t)__ldg(ybar + rb + j); };
        int32_t s0, s1, t0, t1;
        const int32_t pe32 = (int32_t)pe, n32 = (int32_t)n, m32 = (int32_t)m, p32 = (int32_t)p;
        subproblem_of<int32_t>(a_side, pe32, n32, m32, p32, xb, yb, s0, s1, t0, t1);
        a0 = s0; a1 = s1; b0 = t0; b1 = t1;
        chain = a_side ? pe + first_block_at_or_after<int32_t>(m32, p32, xb(pe32))
                       : pe + first_block_at_or_after<int32_t>(n32, p32, yb(pe32));
    } else {
        auto xb = [&](int64_t i) { return __ldg(xbar + rb + i); };
        auto yb = [&](int64_t j) { return __ldg(ybar + rb + j); };
        subproblem_of<int64_t>(a_side, pe, n, m, p, xb, yb, a0, a1, b0, b1);
        chain = a_side ? pe + first_block_at_or_after<int64_t>(m, p, xb(pe))
                       : pe + first_block_at_or_after<int64_t>(n, p, yb(pe));
    }
    TileDesc d{};
    d.a0 = a0g + a0; d.b0 = b0g + b0; d.c0 = c0g + a0 + b0;
    d.nA = (int32_t)(a1 - a0); d.nB = (int32_t)(b1 - b0);
    d.first = chain == 0;
    desc[item_base_of(ps, pb, k) + chain] = d;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

template <typename K>
tm_status launch_engine(const EngineArgs& a, const tm_config* cfg, cudaStream_t s);

struct BatchedWs {
    void* control;
    int64_t* n_items;                              // device record count
    int64_t *search_base, *rank_base, *item_base;  // num_pairs + 1 each (CSR)
    int64_t* part;                                 // 3 x ceil(num_pairs / 256) CTA totals of the scan
    int64_t* cta_pair;                             // pair of each search/plan CTA's first thread (CSR)
    int64_t *xbar, *ybar;
    TileDesc* tiles;
    int4 *ta, *tb;                                 // fused sort rounds: run offsets of every chain point
    Tile4Desc* tiles4;                             // fused sort rounds: four-run records
    size_t bytes;
};

static int64_t tile_of(const tm_config* cfg) { return (cfg && cfg->tile > 0) ? cfg->tile : kDefaultTile; }

// Bounds: p_k <= (n_k + m_k) / tile + 1, so sum p_k <= total / tile + pairs.
static int64_t blocks_bound(int64_t pairs, int64_t total, int64_t tile) { return total / tile + pairs; }

// Workspace: control block, device record count, three per-pair prefix
// arrays, the scan's CTA totals, the first pair of every search/plan CTA,
// cross ranks (ranks_cap entries per side) and tile records.
static BatchedWs ws_layout(void* base, int64_t pairs, int64_t ranks_cap, int64_t items_cap, int64_t ctas_cap,
                           int64_t tuples_cap = 0, int64_t items4_cap = 0) {
    BatchedWs w{};
    uint8_t* b = static_cast<uint8_t*>(base);
    size_t o = 0;
    w.control = b; o += kStatusBytes;
    w.n_items = reinterpret_cast<int64_t*>(b + o); o += 256;
    w.search_base = reinterpret_cast<int64_t*>(b + o); o += align_up((size_t)(pairs + 1) * 8, 256);
    w.rank_base = reinterpret_cast<int64_t*>(b + o); o += align_up((size_t)(pairs + 1) * 8, 256);
    w.item_base = reinterpret_cast<int64_t*>(b + o); o += align_up((size_t)(pairs + 1) * 8, 256);
    w.part = reinterpret_cast<int64_t*>(b + o); o += align_up((size_t)3 * ((pairs + 255) / 256) * 8, 256);
    w.cta_pair = reinterpret_cast<int64_t*>(b + o); o += align_up((size_t)(ctas_cap + 1) * 8, 256);
    w.xbar = reinterpret_cast<int64_t*>(b + o); o += align_up((size_t)ranks_cap * 8, 256);
    w.ybar = reinterpret_cast<int64_t*>(b + o); o += align_up((size_t)ranks_cap * 8, 256);
    w.tiles = reinterpret_cast<TileDesc*>(b + o); o += align_up((size_t)items_cap * sizeof(TileDesc), 256);
    w.ta = reinterpret_cast<int4*>(b + o); o += align_up((size_t)tuples_cap * sizeof(int4), 256);
    w.tb = reinterpret_cast<int4*>(b + o); o += align_up((size_t)tuples_cap * sizeof(int4), 256);
    w.tiles4 = reinterpret_cast<Tile4Desc*>(b + o); o += align_up((size_t)items4_cap * sizeof(Tile4Desc), 256);
    w.bytes = o;
    return w;
}

// CSR pairs: sum (p_k + 1) <= P + pairs and sum items <= 2 P.
static BatchedWs batched_ws_layout(void* base, int64_t pairs, int64_t total, int64_t tile) {
    const int64_t P = blocks_bound(pairs, total, tile);
    return ws_layout(base, pairs, P + pairs, 2 * P, (2 * P + 255) / 256);
}

// Runs search, plan and the engine for a pair set; `ws` laid out as above.
template <typename K>
static tm_status run_pairs(const PairSet& ps, const BatchedWs& w, int64_t total_a, int64_t total_b,
                           const K* A, const void* Av, const K* B, const void* Bv,
                           K* C, void* Cv, int vbytes, int64_t tile, int64_t known_items,
                           const tm_config* cfg, cudaStream_t s) {
    const int64_t total = total_a + total_b;
    PairBases pb{w.search_base, w.rank_base, w.item_base, w.cta_pair};
    int64_t threads;                               // upper bound of sum 2 p_k
    if (ps.scanned()) {
        const int64_t blocks = (ps.num_pairs + 255) / 256;
        pair_count_kernel<<<(unsigned)blocks, 256, 0, s>>>(ps, tile, w.search_base, w.rank_base, w.item_base,
                                                          w.part, blocks);
        part_scan_kernel<<<1, 1024, 0, s>>>(w.part, blocks, ps.num_pairs, w.search_base, w.rank_base,
                                            w.item_base, w.n_items);
        part_add_kernel<<<(unsigned)blocks, 256, 0, s>>>(ps, tile, w.part, blocks, w.search_base, w.rank_base,
                                                         w.item_base, w.cta_pair);
        threads = 2 * blocks_bound(ps.num_pairs, total, tile);
    } else {
        threads = 2 * ps.p_uniform * ps.num_pairs;
    }
    if (const tm_status st_ = launch_status(); st_ != TM_OK) return st_;
    const int64_t grid = (threads + 255) / 256;
    if (grid > 0x7fffffffLL) return TM_ERR_UNSUPPORTED;
    if (grid > 0) {
        batched_search_kernel<K><<<(unsigned)grid, 256, 0, s>>>(ps, pb, A, B, threads, w.xbar, w.ybar);
        batched_plan_kernel<<<(unsigned)grid, 256, 0, s>>>(ps, pb, threads, w.xbar, w.ybar, w.tiles);
    }
    if (const tm_status st_ = launch_status(); st_ != TM_OK) return st_;
    EngineArgs a{};
    a.desc = w.tiles;
    a.n_items = known_items;                       // -1 in CSR mode: read from the device
    a.n_items_dev = w.n_items;
    a.items_bound = known_items >= 0 ? known_items : 2 * blocks_bound(ps.num_pairs, total, tile);
    a.status = static_cast<int32_t*>(w.control);
    a.queue = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(w.control) + 8);
    a.A = A; a.Av = Av; a.lenA = total_a;
    a.B = B; a.Bv = Bv; a.lenB = total_b;
    a.C = C; a.Cv = Cv;
    a.vbytes = vbytes;
    a.cap = (int)(tile + 2);
    if (a.items_bound == 0) return TM_OK;
    return launch_engine<K>(a, cfg, s);
}

template <typename K>
static tm_status batched_typed(int64_t pairs, const int64_t* a_off, const void* a_keys, const uint32_t* a_vals,
                               int64_t total_a, const int64_t* b_off, const void* b_keys, const uint32_t* b_vals,
                               int64_t total_b, void* c_keys, uint32_t* c_vals, void* ws,
                               const tm_config* cfg, cudaStream_t s) {
    const int64_t tile = tile_of(cfg);
    BatchedWs w = batched_ws_layout(ws, pairs, total_a + total_b, tile);
    if (const cudaError_t e_ = cudaMemsetAsync(w.control, 0, 16, s); e_ != cudaSuccess) return cuda_failed(e_);
    if (pairs == 0 || total_a + total_b == 0) return TM_OK;
    PairSet ps{};
    ps.num_pairs = pairs; ps.a_off = a_off; ps.b_off = b_off;
    return run_pairs<K>(ps, w, total_a, total_b, static_cast<const K*>(a_keys), a_vals,
                        static_cast<const K*>(b_keys), b_vals, static_cast<K*>(c_keys), c_vals,
                        payload_size(cfg), tile, -1, cfg, s);
}

// ---------------------------------------------------------------------------
// Stable merge sort (Section 3): stable sorted runs, then merge rounds
// ---------------------------------------------------------------------------

// The stable sorted runs (tm_runsort.cuh): one CTA per run, its keys,
// payloads and digit counts in dynamic shared memory.
template <typename K, typename V>
static tm_status launch_run_sort(unsigned runs, const K* in_k, const V* in_v, K* out_k, V* out_v, int64_t n,
                                 const int64_t* rdesc, cudaStream_t s) {
    if (runs == 0) return TM_OK;
    constexpr uint32_t smem = run_sort_smem_bytes<K, V>();
    if (!ensure_smem_limit(run_sort_kernel<K, V>, smem)) return TM_ERR_UNSUPPORTED;
    run_sort_kernel<K, V><<<runs, kSortThreads, smem, s>>>(in_k, in_v, out_k, out_v, n, rdesc);
    return launch_status();
}

// Pair set of the merge round with sorted runs of length `run`.
static PairSet sort_round(int64_t n, int64_t run, int64_t tile, int64_t* items) {
    PairSet ps{};
    ps.num_pairs = (n + 2 * run - 1) / (2 * run);
    ps.run = run; ps.total = n;
    ps.p_uniform = pair_blocks(run, run, tile);
    const int64_t last_a0 = 2 * (ps.num_pairs - 1) * run;
    const int64_t last_n = n - last_a0 < run ? n - last_a0 : run;
    int64_t last_m = n - last_a0 - last_n < run ? n - last_a0 - last_n : run;
    if (last_m < 0) last_m = 0;
    *items = (ps.num_pairs - 1) * 2 * ps.p_uniform + pair_items(last_n, last_m, ps.p_uniform);
    return ps;
}

// ---------------------------------------------------------------------------
// Two merge-sort rounds fused into one pass: groups of four runs
// ---------------------------------------------------------------------------
// Group q holds runs R_k = X[(4q + k) run, (4q + k + 1) run) (clipped to n),
// k = 0..3.  The pass computes merge(merge(R0, R1), merge(R2, R3)), i.e. the
// outputs of round `run` and of round 2 run, by the paper's method on the
// outer merge of X = merge(R0, R1) and Y = merge(R2, R3): p blocks of each,
// cross ranks of the block starts, the five cases.  X and Y are not stored:
//  * the x-th element of X and the split of R0, R1 it implies come from the
//    co-rank of x in (R0, R1) (the position formulas of Section 2); likewise
//    for Y;
//  * rank_low(v, Y) = rank_low(v, R2) + rank_low(v, R3), and the first
//    rank_low(v, Y) elements of Y are exactly R2[0, rank_low(v, R2)) and
//    R3[0, rank_low(v, R3)); the same holds for rank_high and X.
// So every chain point P_A(i) = (x_i, xbar_i), P_B(j) = (ybar_j, y_j) of the
// outer merge comes with the four run offsets (r0, r1, r2, r3) it splits at,
// and a subproblem between consecutive points is four contiguous ranges.

struct QuadGeom {
    int64_t start[4], len[4];
    int64_t base, nX, nY;
};

__host__ __device__ __forceinline__ QuadGeom quad_geom(int64_t q, int64_t run, int64_t n) {
    QuadGeom g;
    g.base = 4 * q * run;
    for (int k = 0; k < 4; ++k) {
        const int64_t s0 = g.base + k * run, e = s0 + run < n ? s0 + run : n;
        g.start[k] = s0 < n ? s0 : n;
        g.len[k] = e > s0 ? e - s0 : 0;
    }
    g.nX = g.len[0] + g.len[1];
    g.nY = g.len[2] + g.len[3];
    return g;
}

// Number of elements of P (nP) among the first d outputs of the stable
// merge of P and Q (P first on equal keys): the i with Q[d-i-1] < P[i] and
// P[i-1] <= Q[d-i], by bisection in global memory.
template <typename K>
__device__ __forceinline__ int64_t corank_global(const K* __restrict__ P, int64_t nP, const K* __restrict__ Q,
                                                 int64_t nQ, int64_t d) {
    int64_t lo = d > nQ ? d - nQ : 0, hi = d < nP ? d : nP;
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(Q + (d - mid - 1)) < __ldg(P + mid)) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Chain points of every group: thread (q, local): local < p -> A point i
// (block start of X), p <= local < 2p -> B point j (block start of Y),
// local = 2p -> the end points.  xbar / ybar as in Steps 1-2 of the outer
// merge; ta / tb the run offsets of each point.
template <typename K>
__global__ void __launch_bounds__(256)
quad_search_kernel(const K* __restrict__ X, int64_t n, int64_t run, int64_t p, int64_t groups,
                   int64_t* __restrict__ xbar, int64_t* __restrict__ ybar, int4* __restrict__ ta,
                   int4* __restrict__ tb) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t q = div_nonneg<int64_t>(t, 2 * p + 1);
    if (q >= groups) return;
    const int64_t local = t - q * (2 * p + 1);
    const QuadGeom g = quad_geom(q, run, n);
    const K* R0 = X + g.start[0]; const K* R1 = X + g.start[1];
    const K* R2 = X + g.start[2]; const K* R3 = X + g.start[3];
    const int64_t L0 = g.len[0], L1 = g.len[1], L2 = g.len[2], L3 = g.len[3];
    const int64_t pb = q * (p + 1);
    const int4 all = make_int4((int)L0, (int)L1, (int)L2, (int)L3);
    if (local < p) {                                   // A point: block start x of X
        const int64_t i = local, x = block_start<int64_t>(g.nX, p, i);
        if (x >= g.nX) { xbar[pb + i] = g.nY; ta[pb + i] = all; return; }
        const int64_t r0 = corank_global(R0, L0, R1, L1, x), r1 = x - r0;
        const K v = (r1 < L1 && (r0 >= L0 || __ldg(R1 + r1) < __ldg(R0 + r0))) ? __ldg(R1 + r1) : __ldg(R0 + r0);
        const int64_t r2 = rank_low_global<K, int64_t>(R2, L2, v), r3 = rank_low_global<K, int64_t>(R3, L3, v);
        xbar[pb + i] = r2 + r3;
        ta[pb + i] = make_int4((int)r0, (int)r1, (int)r2, (int)r3);
    } else if (local < 2 * p) {                        // B point: block start y of Y
        const int64_t j = local - p, y = block_start<int64_t>(g.nY, p, j);
        if (y >= g.nY) { ybar[pb + j] = g.nX; tb[pb + j] = all; return; }
        const int64_t r2 = corank_global(R2, L2, R3, L3, y), r3 = y - r2;
        const K w = (r3 < L3 && (r2 >= L2 || __ldg(R3 + r3) < __ldg(R2 + r2))) ? __ldg(R3 + r3) : __ldg(R2 + r2);
        const int64_t r0 = rank_high_global<K, int64_t>(R0, L0, w), r1 = rank_high_global<K, int64_t>(R1, L1, w);
        ybar[pb + j] = r0 + r1;
        tb[pb + j] = make_int4((int)r0, (int)r1, (int)r2, (int)r3);
    } else {                                           // the end points (x_p = nX, y_p = nY)
        xbar[pb + p] = g.nY; ybar[pb + p] = g.nX;
        ta[pb + p] = all; tb[pb + p] = all;
    }
}

// Records of every group: the subproblem of each non-empty block of X and
// of Y (the five cases in split-point form, on the outer merge), as the run
// ranges between its chain point and the next one, at its chain index.
__global__ void __launch_bounds__(256)
quad_plan_kernel(int64_t n, int64_t run, int64_t p, int64_t groups, const int64_t* __restrict__ xbar,
                 const int64_t* __restrict__ ybar, const int4* __restrict__ ta, const int4* __restrict__ tb,
                 Tile4Desc* __restrict__ desc, int32_t* status) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t q = div_nonneg<int64_t>(t, 2 * p);
    if (q >= groups) return;
    const int64_t local = t - q * 2 * p;
    const QuadGeom g = quad_geom(q, run, n);
    const bool a_side = local < p;
    const int64_t pe = a_side ? local : local - p;
    if (a_side ? block_start<int64_t>(g.nX, p, pe) >= g.nX : block_start<int64_t>(g.nY, p, pe) >= g.nY) return;
    const int64_t pb = q * (p + 1);
    auto xb = [&](int64_t i) { return __ldg(xbar + pb + i); };
    auto yb = [&](int64_t j) { return __ldg(ybar + pb + j); };
    int64_t a0, a1, b0, b1;
    subproblem_of<int64_t>(a_side, pe, g.nX, g.nY, p, xb, yb, a0, a1, b0, b1);
    // the chain point the subproblem ends at: for an A point the next is
    // P_B(jn) when jn < p and y_jn < xbar_{i+1}, else P_A(i+1) (mirror for B)
    int4 t0, t1;
    int64_t chain;
    if (a_side) {
        const int64_t jn = first_block_at_or_after<int64_t>(g.nY, p, xb(pe));
        t0 = ta[pb + pe];
        t1 = (jn < p && block_start<int64_t>(g.nY, p, jn) < xb(pe + 1)) ? tb[pb + jn] : ta[pb + pe + 1];
        chain = pe + jn;
    } else {
        const int64_t in = first_block_at_or_after<int64_t>(g.nX, p, yb(pe));
        t0 = tb[pb + pe];
        t1 = (in < p && block_start<int64_t>(g.nX, p, in) < yb(pe + 1)) ? ta[pb + in] : tb[pb + pe + 1];
        chain = pe + in;
    }
    Tile4Desc d{};
    // the run offsets must agree with the outer merge's ranges; if not, an
    // empty record (nothing is read) and TM_ERR_BOUNDS
    if ((int64_t)t0.x + t0.y != a0 || (int64_t)t0.z + t0.w != b0 || (int64_t)t1.x + t1.y != a1 ||
        (int64_t)t1.z + t1.w != b1) {
        set_status(status, TM_ERR_BOUNDS);
        for (int k = 0; k < 4; ++k) d.s[k] = g.start[k];
        d.c0 = g.base;
        d.first = chain == 0;
        desc[q * 2 * p + chain] = d;
        return;
    }
    d.s[0] = g.start[0] + t0.x; d.s[1] = g.start[1] + t0.y;
    d.s[2] = g.start[2] + t0.z; d.s[3] = g.start[3] + t0.w;
    d.l[0] = t1.x - t0.x; d.l[1] = t1.y - t0.y; d.l[2] = t1.z - t0.z; d.l[3] = t1.w - t0.w;
    d.c0 = g.base + a0 + b0;
    d.first = chain == 0;
    desc[q * 2 * p + chain] = d;
}

template <typename K>
tm_status launch_engine4(const Engine4Args& a, int vbytes, const tm_config* cfg, cudaStream_t s);

// One fused pair of rounds: runs of `run` sorted in src -> runs of 4 run in dst.
template <typename K>
static tm_status run_quads(const BatchedWs& w, int64_t n, int64_t run, int64_t tile, const K* src,
                           const void* srcv, K* dst, void* dstv, int vbytes, const tm_config* cfg, cudaStream_t s) {
    const int64_t groups = (n + 4 * run - 1) / (4 * run);
    const int64_t p = pair_blocks(2 * run, 2 * run, tile);
    const int64_t threads = groups * (2 * p + 1);
    if ((threads + 255) / 256 > 0x7fffffffLL) return TM_ERR_UNSUPPORTED;
    quad_search_kernel<K><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(src, n, run, p, groups, w.xbar,
                                                                           w.ybar, w.ta, w.tb);
    quad_plan_kernel<<<(unsigned)((groups * 2 * p + 255) / 256), 256, 0, s>>>(
        n, run, p, groups, w.xbar, w.ybar, w.ta, w.tb, w.tiles4, static_cast<int32_t*>(w.control));
    if (const tm_status st_ = launch_status(); st_ != TM_OK) return st_;
    // records: every group but the last has 2p; the last has one per
    // non-empty block of its X and of its Y
    const QuadGeom gl = quad_geom(groups - 1, run, n);
    const int64_t items = (groups - 1) * 2 * p + pair_items(gl.nX, gl.nY, p);
    Engine4Args a{};
    a.desc = w.tiles4;
    a.n_items = items;
    a.queue = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(w.control) + 8);
    a.status = static_cast<int32_t*>(w.control);
    a.src = src; a.srcv = srcv; a.len = n;
    a.C = dst; a.Cv = dstv;
    a.cap = (int)(tile + 2);
    return launch_engine4<K>(a, vbytes, cfg, s);
}

// Whether the sort fuses pairs of rounds: cfg->merge_ways = 4 asks for it;
// the four-run engine takes the diagonal in-CTA split only and tiles up to
// 4606 elements (9-element runs of its 512 consumer threads).
static bool sort_fuses(const tm_config* cfg, int64_t tile) {
    if (!cfg || cfg->merge_ways != 4 || cfg->split == TM_SPLIT_BLOCKS) return false;
    return tile + 2 <= 9 * 512;
}

// The largest rank, tuple and record counts over all merge rounds.
static BatchedWs sort_ws_layout(void* base, int64_t n, int64_t tile) {
    int64_t ranks = 0, items = 0, tuples = 0, items4 = 0;
    for (int64_t run = kSortRun; run < n; run *= 2) {
        int64_t it = 0;
        PairSet ps = sort_round(n, run, tile, &it);
        const int64_t r = ps.num_pairs * (ps.p_uniform + 1);
        if (r > ranks) ranks = r;
        if (2 * ps.num_pairs * ps.p_uniform > items) items = 2 * ps.num_pairs * ps.p_uniform;
        const int64_t groups = (n + 4 * run - 1) / (4 * run), p4 = pair_blocks(2 * run, 2 * run, tile);
        if (groups * (p4 + 1) > tuples) tuples = groups * (p4 + 1);
        if (groups * 2 * p4 > items4) items4 = groups * 2 * p4;
    }
    if (tuples > ranks) ranks = tuples;
    return ws_layout(base, 0, ranks, items, 0, tuples, items4);
}

template <typename K, typename V>
static tm_status sort_typed_v(void* keys, void* vals, int64_t n, void* tmp_keys, void* tmp_vals,
                              void* ws, const tm_config* cfg, cudaStream_t s) {
    const int64_t tile = tile_of(cfg);
    BatchedWs w = sort_ws_layout(ws, n, tile);
    if (const cudaError_t e_ = cudaMemsetAsync(w.control, 0, 16, s); e_ != cudaSuccess) return cuda_failed(e_);
    if (n <= 1) return TM_OK;
    K* bufk[2] = {static_cast<K*>(keys), static_cast<K*>(tmp_keys)};
    V* bufv[2] = {static_cast<V*>(vals), static_cast<V*>(tmp_vals)};
    // pairwise rounds (run 4096, 8192, ...), fused two at a time when the
    // configuration allows; the number of passes decides where the run
    // formation writes, so that the last pass lands in (keys, vals)
    int rounds = 0;
    for (int64_t r = kSortRun; r < n; r *= 2) ++rounds;
    // fused pairs while two rounds remain and the runs' offsets fit int32
    int fused = 0;
    if (sort_fuses(cfg, tile))
        for (int64_t r = kSortRun; rounds - 2 * fused >= 2 && r <= (1LL << 29); r *= 4) ++fused;
    const int passes = fused + (rounds - 2 * fused);
    int src = (passes % 2 == 0) ? 0 : 1;
    const int64_t runs = (n + kSortRun - 1) / kSortRun;
    if (runs > 0x7fffffffLL) return TM_ERR_UNSUPPORTED;
    if (const tm_status st_ = launch_run_sort<K, V>((unsigned)runs, bufk[0], bufv[0], bufk[src], bufv[src], n,
                                                     nullptr, s); st_ != TM_OK) return st_;
    int64_t run = kSortRun;
    for (int f = 0; f < fused; ++f, run *= 4) {
        const int dst = src ^ 1;
        tm_status st = run_quads<K>(w, n, run, tile, bufk[src], vals ? bufv[src] : nullptr, bufk[dst],
                                    vals ? bufv[dst] : nullptr, (int)sizeof(V), cfg, s);
        if (st != TM_OK) return st;
        src = dst;
    }
    for (; run < n; run *= 2) {
        int64_t items = 0;
        const PairSet ps = sort_round(n, run, tile, &items);
        const int dst = src ^ 1;
        tm_status st = run_pairs<K>(ps, w, n, n, bufk[src], bufv[src], bufk[src], bufv[src],
                                    bufk[dst], bufv[dst], (int)sizeof(V), tile, items, cfg, s);
        if (st != TM_OK) return st;
        src = dst;
    }
    return TM_OK;
}

template <typename K>
static tm_status sort_typed(void* keys, uint32_t* vals, int64_t n, void* tmp_keys, uint32_t* tmp_vals,
                            void* ws, const tm_config* cfg, cudaStream_t s) {
    if (payload_size(cfg) == 8) return sort_typed_v<K, uint64_t>(keys, vals, n, tmp_keys, tmp_vals, ws, cfg, s);
    return sort_typed_v<K, uint32_t>(keys, vals, n, tmp_keys, tmp_vals, ws, cfg, s);
}

// ---------------------------------------------------------------------------
// Segmented stable merge sort: independent segments of one array
// ---------------------------------------------------------------------------
// Runs of at most kSortRun elements inside each segment (a run never
// crosses a segment boundary), then rounds of width w = kSortRun,
// 2 kSortRun, ...: in every round each segment's neighbouring runs are
// merged pairwise (a last unpaired run, or a segment already sorted, is a
// pair with an empty second run: a copy).  The plan is made on the host from the host's segment
// offsets; every round is one batched merge over explicit pairs.

struct SegPlan {
    int64_t segs = 0, runs = 0;
    std::vector<int64_t> round_pairs;   // pairs of every round
    int64_t max_pairs = 0;
};

// false when the offsets are not 0 = off[0] <= ... <= off[segs] = n.
static bool seg_plan(const int64_t* off, int64_t segs, int64_t n, SegPlan& P) {
    if (segs < 0 || (segs > 0 && off == nullptr)) return false;
    if (segs == 0) return n == 0;
    if (off[0] != 0 || off[segs] != n) return false;
    int64_t maxlen = 0;
    P.segs = segs;
    for (int64_t q = 0; q < segs; ++q) {
        const int64_t len = off[q + 1] - off[q];
        if (len < 0) return false;
        maxlen = len > maxlen ? len : maxlen;
        P.runs += (len + kSortRun - 1) / kSortRun;
    }
    for (int64_t w = kSortRun; w < maxlen; w *= 2) {
        int64_t cnt = 0;
        for (int64_t q = 0; q < segs; ++q) cnt += (off[q + 1] - off[q] + 2 * w - 1) / (2 * w);
        P.round_pairs.push_back(cnt);
        if (cnt > P.max_pairs) P.max_pairs = cnt;
    }
    return true;
}

// Exclusive prefix over the segments of ceil(len_q / unit) (one CTA,
// rounds of 1024 with a running carry); pre[segs] = the total.
__global__ void __launch_bounds__(1024)
seg_prefix_kernel(const int64_t* __restrict__ off, int64_t segs, int64_t unit, int64_t* __restrict__ pre) {
    int64_t carry = 0;
    for (int64_t r = 0; r < segs; r += 1024) {
        const int64_t q = r + threadIdx.x;
        int64_t v[3] = {q < segs ? (off[q + 1] - off[q] + unit - 1) / unit : 0, 0, 0};
        int64_t ex[3], tot[3];
        block_scan3<1024>(v, ex, tot);
        if (q < segs) pre[q] = carry + ex[0];
        carry += tot[0];
    }
    if (threadIdx.x == 0) pre[segs] = carry;
}

// Runs of segment q: (start, length) at pre[q]...; thread per segment.
__global__ void __launch_bounds__(256)
seg_runs_kernel(const int64_t* __restrict__ off, int64_t segs, const int64_t* __restrict__ pre,
                int64_t* __restrict__ rdesc) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= segs) return;
    int64_t o = pre[q];
    for (int64_t a = off[q]; a < off[q + 1]; a += kSortRun, ++o) {
        rdesc[2 * o] = a;
        rdesc[2 * o + 1] = off[q + 1] - a < kSortRun ? off[q + 1] - a : kSortRun;
    }
}

// Pairs of segment q in the round of width w: (a0, n, m) at pre[q]...
__global__ void __launch_bounds__(256)
seg_pairs_kernel(const int64_t* __restrict__ off, int64_t segs, int64_t w, const int64_t* __restrict__ pre,
                 int64_t* __restrict__ pdesc) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= segs) return;
    int64_t o = pre[q];
    for (int64_t a0 = off[q]; a0 < off[q + 1]; a0 += 2 * w, ++o) {
        const int64_t na = off[q + 1] - a0 < w ? off[q + 1] - a0 : w;
        const int64_t rest = off[q + 1] - a0 - na;
        pdesc[3 * o] = a0;
        pdesc[3 * o + 1] = na;
        pdesc[3 * o + 2] = rest < w ? rest : w;
    }
}

// Workspace: the batched layout for the largest round, then the segment
// offsets, a prefix array, the run and the pair descriptors.
struct SegWs { BatchedWs w; int64_t *off, *pre, *rd, *pd; };

static SegWs seg_ws_layout(void* base, const SegPlan& P, int64_t n, int64_t tile) {
    SegWs x;
    x.w = batched_ws_layout(base, P.max_pairs, 2 * n, tile);
    uint8_t* b = static_cast<uint8_t*>(base);
    size_t o = x.w.bytes;
    x.off = reinterpret_cast<int64_t*>(b + o); o += align_up((size_t)(P.segs + 1) * 8, 256);
    x.pre = reinterpret_cast<int64_t*>(b + o); o += align_up((size_t)(P.segs + 1) * 8, 256);
    x.rd = reinterpret_cast<int64_t*>(b + o); o += align_up((size_t)P.runs * 16, 256);
    x.pd = reinterpret_cast<int64_t*>(b + o); o += align_up((size_t)P.max_pairs * 24, 256);
    x.w.bytes = o;
    return x;
}

template <typename K, typename V>
static tm_status sort_segmented_v(void* keys, void* vals, int64_t n, void* tmp_keys, void* tmp_vals,
                                  const int64_t* host_off, const SegPlan& P, void* ws, const tm_config* cfg,
                                  cudaStream_t s) {
    const int64_t tile = tile_of(cfg);
    SegWs x = seg_ws_layout(ws, P, n, tile);
    BatchedWs& w = x.w;
    if (const cudaError_t e_ = cudaMemsetAsync(w.control, 0, 16, s); e_ != cudaSuccess) return cuda_failed(e_);
    if (n == 0) return TM_OK;
    // the segment offsets (pageable host memory, staged before the call returns)
    if (const cudaError_t e_ = cudaMemcpyAsync(x.off, host_off, (size_t)(P.segs + 1) * 8, cudaMemcpyHostToDevice, s);
        e_ != cudaSuccess)
        return cuda_failed(e_);
    const unsigned sg = (unsigned)((P.segs + 255) / 256);
    seg_prefix_kernel<<<1, 1024, 0, s>>>(x.off, P.segs, kSortRun, x.pre);
    seg_runs_kernel<<<sg, 256, 0, s>>>(x.off, P.segs, x.pre, x.rd);
    if (const tm_status st_ = launch_status(); st_ != TM_OK) return st_;
    K* bufk[2] = {static_cast<K*>(keys), static_cast<K*>(tmp_keys)};
    V* bufv[2] = {static_cast<V*>(vals), static_cast<V*>(tmp_vals)};
    const int rounds = (int)P.round_pairs.size();
    int src = (rounds % 2 == 0) ? 0 : 1;
    if (P.runs > 0x7fffffffLL) return TM_ERR_UNSUPPORTED;
    if (const tm_status st_ = launch_run_sort<K, V>((unsigned)P.runs, bufk[0], bufv[0], bufk[src], bufv[src], n,
                                                     x.rd, s); st_ != TM_OK) return st_;
    int64_t wd = kSortRun;
    for (int r = 0; r < rounds; ++r, wd *= 2) {
        seg_prefix_kernel<<<1, 1024, 0, s>>>(x.off, P.segs, 2 * wd, x.pre);
        seg_pairs_kernel<<<sg, 256, 0, s>>>(x.off, P.segs, wd, x.pre, x.pd);
        if (const tm_status st_ = launch_status(); st_ != TM_OK) return st_;
        PairSet ps{};
        ps.num_pairs = P.round_pairs[r];
        ps.pdesc = x.pd;
        const int dst = src ^ 1;
        tm_status st = run_pairs<K>(ps, w, n, n, bufk[src], bufv[src], bufk[src], bufv[src], bufk[dst], bufv[dst],
                                    (int)sizeof(V), tile, -1, cfg, s);
        if (st != TM_OK) return st;
        src = dst;
    }
    return TM_OK;
}

template <typename K>
static tm_status sort_segmented_typed(void* keys, uint32_t* vals, int64_t n, void* tmp_keys, uint32_t* tmp_vals,
                                      const int64_t* off, const SegPlan& P, void* ws, const tm_config* cfg,
                                      cudaStream_t s) {
    if (payload_size(cfg) == 8)
        return sort_segmented_v<K, uint64_t>(keys, vals, n, tmp_keys, tmp_vals, off, P, ws, cfg, s);
    return sort_segmented_v<K, uint32_t>(keys, vals, n, tmp_keys, tmp_vals, off, P, ws, cfg, s);
}

// ---------------------------------------------------------------------------
// Autotuner: times candidate configurations on the caller's data with CUDA
// events and remembers the fastest per (key type, size bucket, operation).
// ---------------------------------------------------------------------------

struct TuneKey {
    int op, kt, vbytes, log2_total;
    bool operator<(const TuneKey& o) const {
        return std::tie(op, kt, vbytes, log2_total) < std::tie(o.op, o.kt, o.vbytes, o.log2_total);
    }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, tm_config> g_tune;

static int log2_bucket(int64_t x) { int b = 0; while ((int64_t(1) << (b + 1)) <= x) ++b; return b; }

// The autotuned configuration for a call whose cfg is NULL or sets nothing
// but the payload width.
static bool tuned_config(int op, tm_key_type kt, int64_t total, const tm_config* cfg, tm_config* out) {
    if (cfg) {
        tm_config d{};
        d.payload_bytes = cfg->payload_bytes;
        if (std::memcmp(&d, cfg, sizeof(tm_config)) != 0) return false;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(TuneKey{op, (int)kt, payload_size(cfg), log2_bucket(total)});
    if (it == g_tune.end()) return false;
    *out = it->second;
    return true;
}

}  // namespace pmerge

using namespace pmerge;

namespace {
tm_status check_batched(tm_key_type kt, int64_t pairs, const int64_t* a_off, const void* a_keys,
                        const uint32_t* a_vals, int64_t total_a, const int64_t* b_off, const void* b_keys,
                        const uint32_t* b_vals, int64_t total_b, void* c_keys, uint32_t* c_vals, int vsize) {
    if (pairs < 0 || total_a < 0 || total_b < 0) return TM_ERR_INVALID;
    if (kt < TM_KEY_U32 || kt > TM_KEY_F32 || vsize < 0) return TM_ERR_UNSUPPORTED;
    const size_t E = key_size(kt);
    if (pairs > 0 && (!aligned(a_off, 8) || !aligned(b_off, 8))) return TM_ERR_INVALID;
    if ((total_a > 0 && !aligned(a_keys, E)) || (total_b > 0 && !aligned(b_keys, E)) ||
        (total_a + total_b > 0 && !aligned(c_keys, E)) ||
        !payloads_ok(total_a, a_vals, total_b, b_vals, c_vals, vsize))
        return TM_ERR_INVALID;
    return TM_OK;
}

tm_status batched_dispatch(tm_key_type kt, int64_t pairs, const int64_t* a_off, const void* a_keys,
                           const uint32_t* a_vals, int64_t total_a, const int64_t* b_off, const void* b_keys,
                           const uint32_t* b_vals, int64_t total_b, void* c_keys, uint32_t* c_vals,
                           void* ws, const tm_config* cfg, cudaStream_t s) {
    switch (kt) {
        case TM_KEY_U32: return batched_typed<uint32_t>(pairs, a_off, a_keys, a_vals, total_a, b_off, b_keys, b_vals, total_b, c_keys, c_vals, ws, cfg, s);
        case TM_KEY_I32: return batched_typed<int32_t>(pairs, a_off, a_keys, a_vals, total_a, b_off, b_keys, b_vals, total_b, c_keys, c_vals, ws, cfg, s);
        case TM_KEY_U64: return batched_typed<uint64_t>(pairs, a_off, a_keys, a_vals, total_a, b_off, b_keys, b_vals, total_b, c_keys, c_vals, ws, cfg, s);
        case TM_KEY_F32: return batched_typed<float>(pairs, a_off, a_keys, a_vals, total_a, b_off, b_keys, b_vals, total_b, c_keys, c_vals, ws, cfg, s);
    }
    return TM_ERR_UNSUPPORTED;
}
}  // namespace

extern "C" {

size_t tm_merge_batched_workspace_size(int64_t num_pairs, int64_t total_a, int64_t total_b, const tm_config* cfg) {
    if (num_pairs < 0 || total_a < 0 || total_b < 0) return 0;
    return batched_ws_layout(nullptr, num_pairs, total_a + total_b, tile_of(cfg)).bytes;
}

tm_status tm_merge_batched(tm_key_type kt, int64_t num_pairs,
                           const int64_t* a_offsets, const void* a_keys, const uint32_t* a_vals, int64_t total_a,
                           const int64_t* b_offsets, const void* b_keys, const uint32_t* b_vals, int64_t total_b,
                           void* c_keys, uint32_t* c_vals, void* workspace, size_t workspace_bytes,
                           const tm_config* cfg, tm_stream_t stream) {
    tm_status st = check_batched(kt, num_pairs, a_offsets, a_keys, a_vals, total_a, b_offsets, b_keys, b_vals,
                                 total_b, c_keys, c_vals, payload_size(cfg));
    if (st != TM_OK) return st;
    tm_config tuned;
    if (tuned_config(1, kt, total_a + total_b, cfg, &tuned)) cfg = &tuned;
    if (!workspace || !aligned(workspace, 256) ||
        workspace_bytes < tm_merge_batched_workspace_size(num_pairs, total_a, total_b, cfg))
        return TM_ERR_WORKSPACE;
    return batched_dispatch(kt, num_pairs, a_offsets, a_keys, a_vals, total_a, b_offsets, b_keys, b_vals,
                            total_b, c_keys, c_vals, workspace, cfg, reinterpret_cast<cudaStream_t>(stream));
}

size_t tm_merge_sort_workspace_size(int64_t n, const tm_config* cfg) {
    if (n < 0) return 0;
    return sort_ws_layout(nullptr, n, tile_of(cfg)).bytes;
}

tm_status tm_merge_sort(tm_key_type kt, void* keys, uint32_t* vals, int64_t n, void* tmp_keys, uint32_t* tmp_vals,
                        void* workspace, size_t workspace_bytes, const tm_config* cfg, tm_stream_t stream) {
    if (n < 0) return TM_ERR_INVALID;
    const int vs = payload_size(cfg);
    if (kt < TM_KEY_U32 || kt > TM_KEY_F32 || vs < 0) return TM_ERR_UNSUPPORTED;
    if (cfg && cfg->merge_ways != 0 && cfg->merge_ways != 2 && cfg->merge_ways != 4) return TM_ERR_UNSUPPORTED;
    const size_t E = key_size(kt);
    if (n > 0 && (!aligned(keys, E) || !aligned(tmp_keys, E) ||
                  ((vals || tmp_vals) && (!aligned(vals, vs) || !aligned(tmp_vals, vs)))))
        return TM_ERR_INVALID;                      // vals and tmp_vals both NULL: keys only
    tm_config tuned;
    if (tuned_config(2, kt, n, cfg, &tuned)) cfg = &tuned;
    if (!workspace || !aligned(workspace, 256) || workspace_bytes < tm_merge_sort_workspace_size(n, cfg))
        return TM_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (kt) {
        case TM_KEY_U32: return sort_typed<uint32_t>(keys, vals, n, tmp_keys, tmp_vals, workspace, cfg, s);
        case TM_KEY_I32: return sort_typed<int32_t>(keys, vals, n, tmp_keys, tmp_vals, workspace, cfg, s);
        case TM_KEY_U64: return sort_typed<uint64_t>(keys, vals, n, tmp_keys, tmp_vals, workspace, cfg, s);
        case TM_KEY_F32: return sort_typed<float>(keys, vals, n, tmp_keys, tmp_vals, workspace, cfg, s);
    }
    return TM_ERR_UNSUPPORTED;
}

size_t tm_merge_sort_segmented_workspace_size(int64_t n, const int64_t* seg_offsets, int64_t num_segments,
                                              const tm_config* cfg) {
    SegPlan P;
    if (n < 0 || !seg_plan(seg_offsets, num_segments, n, P)) return 0;
    return seg_ws_layout(nullptr, P, n, tile_of(cfg)).w.bytes;
}

tm_status tm_merge_sort_segmented(tm_key_type kt, void* keys, uint32_t* vals, int64_t n,
                                  const int64_t* seg_offsets, int64_t num_segments, void* tmp_keys,
                                  uint32_t* tmp_vals, void* workspace, size_t workspace_bytes, const tm_config* cfg,
                                  tm_stream_t stream) {
    if (n < 0) return TM_ERR_INVALID;
    const int vs = payload_size(cfg);
    if (kt < TM_KEY_U32 || kt > TM_KEY_F32 || vs < 0) return TM_ERR_UNSUPPORTED;
    const size_t E = key_size(kt);
    if (n > 0 && (!aligned(keys, E) || !aligned(tmp_keys, E) ||
                  ((vals || tmp_vals) && (!aligned(vals, vs) || !aligned(tmp_vals, vs)))))
        return TM_ERR_INVALID;
    SegPlan P;
    if (!seg_plan(seg_offsets, num_segments, n, P)) return TM_ERR_INVALID;
    if (!workspace || !aligned(workspace, 256) ||
        workspace_bytes < seg_ws_layout(nullptr, P, n, tile_of(cfg)).w.bytes)
        return TM_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (kt) {
        case TM_KEY_U32: return sort_segmented_typed<uint32_t>(keys, vals, n, tmp_keys, tmp_vals, seg_offsets, P, workspace, cfg, s);
        case TM_KEY_I32: return sort_segmented_typed<int32_t>(keys, vals, n, tmp_keys, tmp_vals, seg_offsets, P, workspace, cfg, s);
        case TM_KEY_U64: return sort_segmented_typed<uint64_t>(keys, vals, n, tmp_keys, tmp_vals, seg_offsets, P, workspace, cfg, s);
        case TM_KEY_F32: return sort_segmented_typed<float>(keys, vals, n, tmp_keys, tmp_vals, seg_offsets, P, workspace, cfg, s);
    }
    return TM_ERR_UNSUPPORTED;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner
// ---------------------------------------------------------------------------

namespace {

// Candidate configurations: tile x consumer threads x input stages (the
// diagonal in-CTA split).  Each is run once to warm up and once timed.
std::vector<tm_config> tune_candidates() {
    std::vector<tm_config> c;
    const int tiles[] = {1024, 2048, 4096};
    const int threads[] = {128, 256};
    const int stages[] = {3, 4};
    for (int t : tiles)
        for (int th : threads)
            for (int st : stages) {
                tm_config x{};
                x.tile = t; x.threads = th; x.stages = st; x.split = TM_SPLIT_DIAGONAL;
                c.push_back(x);
            }
    return c;
}

template <typename Run>
tm_status tune(int op, tm_key_type kt, int vbytes, int64_t total, size_t ws_have,
               size_t (*ws_need)(const tm_config*), Run run, tm_config* best_out, cudaStream_t s) {
    cudaEvent_t e0, e1;
    if (const cudaError_t e = cudaEventCreate(&e0); e != cudaSuccess) return cuda_failed(e);
    if (const cudaError_t e = cudaEventCreate(&e1); e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_failed(e);
    }
    float best_ms = -1.f;
    tm_config best{};
    for (tm_config c : tune_candidates()) {
        c.payload_bytes = vbytes;
        if (ws_need(&c) > ws_have) continue;
        if (run(&c) != TM_OK) continue;                   // warm-up (and support check)
        cudaEventRecord(e0, s);
        tm_status st = run(&c);
        cudaEventRecord(e1, s);
        if (st != TM_OK || cudaEventSynchronize(e1) != cudaSuccess) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best_ms < 0.f || ms < best_ms) { best_ms = ms; best = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms < 0.f) return TM_ERR_UNSUPPORTED;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[TuneKey{op, (int)kt, vbytes, log2_bucket(total)}] = best;
    }
    if (best_out) *best_out = best;
    return TM_OK;
}

thread_local int64_t t_pairs, t_total_a, t_total_b, t_n;
size_t batched_ws_need(const tm_config* c) { return tm_merge_batched_workspace_size(t_pairs, t_total_a, t_total_b, c); }
size_t sort_ws_need(const tm_config* c) { return tm_merge_sort_workspace_size(t_n, c); }

}  // namespace

extern "C" {

tm_status tm_autotune_batched(tm_key_type kt, int64_t num_pairs,
                              const int64_t* a_offsets, const void* a_keys, const uint32_t* a_vals, int64_t total_a,
                              const int64_t* b_offsets, const void* b_keys, const uint32_t* b_vals, int64_t total_b,
                              void* c_keys, uint32_t* c_vals, void* workspace, size_t workspace_bytes,
                              tm_config* best, tm_stream_t stream) {
    const int vb = best ? payload_size(best) : 4;      // *best on input: the payload width of the trials
    tm_status st = check_batched(kt, num_pairs, a_offsets, a_keys, a_vals, total_a, b_offsets, b_keys, b_vals,
                                 total_b, c_keys, c_vals, vb);
    if (st != TM_OK) return st;
    if (!workspace || !aligned(workspace, 256)) return TM_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    t_pairs = num_pairs; t_total_a = total_a; t_total_b = total_b;
    auto run = [&](const tm_config* c) {
        return batched_dispatch(kt, num_pairs, a_offsets, a_keys, a_vals, total_a, b_offsets, b_keys, b_vals,
                                total_b, c_keys, c_vals, workspace, c, s);
    };
    return tune(1, kt, vb, total_a + total_b, workspace_bytes, batched_ws_need, run, best, s);
}

tm_status tm_autotune_sort(tm_key_type kt, const void* src_keys, const uint32_t* src_vals, int64_t n,
                           void* keys, uint32_t* vals, void* tmp_keys, uint32_t* tmp_vals,
                           void* workspace, size_t workspace_bytes, tm_config* best, tm_stream_t stream) {
    if (n < 0) return TM_ERR_INVALID;
    const int vb = best ? payload_size(best) : 4;      // *best on input: the payload width of the trials
    if (kt < TM_KEY_U32 || kt > TM_KEY_F32 || vb < 0) return TM_ERR_UNSUPPORTED;
    const size_t E = key_size(kt);
    if (n > 0 && (!aligned(src_keys, E) || !aligned(keys, E) || !aligned(tmp_keys, E) ||
                  ((src_vals || vals || tmp_vals) &&
                   (!aligned(src_vals, vb) || !aligned(vals, vb) || !aligned(tmp_vals, vb)))))
        return TM_ERR_INVALID;
    if (!workspace || !aligned(workspace, 256)) return TM_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    t_n = n;
    // every trial sorts a fresh copy of the source; the copy is outside the
    // timed sort only in the sense that it is the same for every candidate
    auto run = [&](const tm_config* c) -> tm_status {
        cudaError_t e = cudaMemcpyAsync(keys, src_keys, (size_t)n * E, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && vals)                 // keys-only sort: no payloads to copy
            e = cudaMemcpyAsync(vals, src_vals, (size_t)n * vb, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_failed(e);
        return tm_merge_sort(kt, keys, vals, n, tmp_keys, tmp_vals, workspace, workspace_bytes, c, stream);
    };
    return tune(2, kt, vb, n, workspace_bytes, sort_ws_need, run, best, s);
}

int tm_autotune_clear(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const int k = (int)g_tune.size();
    g_tune.clear();
    return k;
}

// ---------------------------------------------------------------------------
// CUDA graphs: capture any sequence of calls on a stream, replay it
// ---------------------------------------------------------------------------

struct tm_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

tm_status tm_graph_capture_begin(tm_stream_t stream) {
    if (!stream) return TM_ERR_INVALID;              // the legacy stream cannot be captured
    const cudaError_t e = cudaStreamBeginCapture(reinterpret_cast<cudaStream_t>(stream),
                                                 cudaStreamCaptureModeThreadLocal);
    return e == cudaSuccess ? TM_OK : cuda_failed(e);
}

tm_status tm_graph_capture_end(tm_stream_t stream, tm_graph** out) {
    if (!stream || !out) return TM_ERR_INVALID;
    *out = nullptr;
    cudaGraph_t g = nullptr;
    if (const cudaError_t err = cudaStreamEndCapture(reinterpret_cast<cudaStream_t>(stream), &g);
        err != cudaSuccess || !g)
        return cuda_failed(err != cudaSuccess ? err : cudaErrorStreamCaptureInvalidated);
    cudaGraphExec_t e = nullptr;
    if (const cudaError_t err = cudaGraphInstantiate(&e, g, 0); err != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_failed(err);
    }
    tm_graph* h = new (std::nothrow) tm_graph{g, e};
    if (!h) {
        cudaGraphExecDestroy(e);
        cudaGraphDestroy(g);
        return TM_ERR_INVALID;
    }
    *out = h;
    return TM_OK;
}

tm_status tm_graph_launch(tm_graph* g, tm_stream_t stream) {
    if (!g) return TM_ERR_INVALID;
    const cudaError_t e = cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? TM_OK : cuda_failed(e);
}

void tm_graph_destroy(tm_graph* g) {
    if (!g) return;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
}

}  // extern "C"
