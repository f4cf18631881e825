// Single stable merge (Section 2): the cross-rank search kernel (Steps 1-2)
// and the staged tile-merge kernel (Steps 3-4), plus their C-ABI entry
// points.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "tm_engine.cuh"
#include "tm_host.h"
#include "tm_tile.cuh"

namespace pmerge {

// TM_OK, or TM_ERR_CUDA with the pending launch error recorded for
// tm_last_cuda_error.
static tm_status launch_status() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TM_OK : cuda_failed(e);
}

static thread_local cudaError_t g_last_cuda_error = cudaSuccess;
void record_cuda_error(cudaError_t e) { g_last_cuda_error = e; }
static cudaError_t last_cuda_error() { return g_last_cuda_error; }

// ---------------------------------------------------------------------------
// Steps 1-2: cross-rank search kernel
// ---------------------------------------------------------------------------
// Thread t < p:      xbar[t] = rank_low(A[x_t], B)      (x_t = n -> m)
// Thread p + t:      ybar[t] = rank_high(B[y_t], A)     (y_t = m -> n)
// Thread 2p:         xbar[p] = m, ybar[p] = n.
// Each search is ceil(log2(len + 1)) dependent probes; the probes of
// neighbouring threads share the upper levels of the search tree in L2.
template <typename K>
__global__ void __launch_bounds__(256)
cross_rank_kernel(const K* __restrict__ A, int64_t n, const K* __restrict__ B, int64_t m,
                  int64_t p, int64_t* __restrict__ xbar, int64_t* __restrict__ ybar) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < p) {                        // B-block starts first: with m <= n theirs are the longer searches
        int64_t yj = block_start<int64_t>(m, p, t);
        ybar[t] = (yj < m) ? rank_high_global<K, int64_t>(A, n, __ldg(B + yj)) : n;
    } else if (t < 2 * p) {
        int64_t i = t - p;
        int64_t xi = block_start<int64_t>(n, p, i);
        xbar[i] = (xi < n) ? rank_low_global<K, int64_t>(B, m, __ldg(A + xi)) : m;
    } else if (t == 2 * p) {
        xbar[p] = m;
        ybar[p] = n;
    }
}

template <typename K>
__global__ void __launch_bounds__(256)
rank_search_kernel(const K* __restrict__ q, int64_t count, const K* __restrict__ X, int64_t len,
                   int kind, int64_t* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    K x = __ldg(q + t);
    out[t] = kind ? rank_high_global<K, int64_t>(X, len, x) : rank_low_global<K, int64_t>(X, len, x);
}

__global__ void __launch_bounds__(256)
subproblem_table_kernel(int64_t n, int64_t m, int64_t p, const int64_t* __restrict__ xbar,
                        const int64_t* __restrict__ ybar, int64_t* __restrict__ table) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2 * p) return;
    auto xb = [&](int64_t i) { return xbar[i]; };
    auto yb = [&](int64_t j) { return ybar[j]; };
    int64_t a0, a1, b0, b1;
    subproblem_of<int64_t>(k < p, k < p ? k : k - p, n, m, p, xb, yb, a0, a1, b0, b1);
    table[4 * k + 0] = a0; table[4 * k + 1] = a1;
    table[4 * k + 2] = b0; table[4 * k + 3] = b1;
}

// Steps 3-4 planning: one thread per processing element writes the tile
// record of its subproblem (the split-point form of the five cases) at the
// subproblem's place on the merge path.  A point P_A(i) = (x_i, xbar_i) has
// i A-points and first_block_at_or_after(m, p, xbar_i) B-points before it
// (B block j starts before A[x_i] iff y_j < xbar_i), and symmetrically for
// P_B(j); so the chain index is a sum of two O(1) terms.  Empty blocks (when
// p exceeds a length) have empty subproblems and write nothing; the
// non-empty records fill indices [0, min(p, n) + min(p, m)).
__global__ void __launch_bounds__(256)
plan_single_kernel(int64_t n, int64_t m, int64_t p, const int64_t* __restrict__ xbar,
                   const int64_t* __restrict__ ybar, TileDesc* __restrict__ desc) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2 * p) return;
    auto xb = [&](int64_t i) { return __ldg(xbar + i); };
    auto yb = [&](int64_t j) { return __ldg(ybar + j); };
    plan_single_record(n, m, p, k, xb, yb, desc);
}

// ---------------------------------------------------------------------------
// Ablation: equal-output partitioning (prior work, Section 1) instead of the
// paper's blocks.  Cut k sits at output diagonal d_k = min(k * tile, n + m);
// its co-rank is the number of A elements among the first d_k outputs of the
// stable merge, the i with B[d-i-1] < A[i] and A[i-1] <= B[d-i] (the position
// formulas of Section 2), found by bisection along the diagonal.
// ---------------------------------------------------------------------------

template <typename K>
__global__ void __launch_bounds__(256)
diagonal_corank_kernel(const K* __restrict__ A, int64_t n, const K* __restrict__ B, int64_t m, int64_t tile,
                       int64_t cuts, int64_t* __restrict__ corank) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k > cuts) return;
    const int64_t d = k * tile < n + m ? k * tile : n + m;
    int64_t lo = d > m ? d - m : 0, hi = d < n ? d : n;
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(B + (d - mid - 1)) < __ldg(A + mid)) hi = mid; else lo = mid + 1;
    }
    corank[k] = lo;
}

// One record per output range [d_k, d_k+1): tile elements each (the last
// fewer), never packed.
__global__ void __launch_bounds__(256)
diagonal_plan_kernel(int64_t n, int64_t m, int64_t tile, int64_t cuts, const int64_t* __restrict__ corank,
                     TileDesc* __restrict__ desc) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cuts) return;
    const int64_t d0 = k * tile, d1 = (k + 1) * tile < n + m ? (k + 1) * tile : n + m;
    const int64_t i0 = __ldg(corank + k), i1 = __ldg(corank + k + 1);
    TileDesc d{};
    d.a0 = i0; d.b0 = d0 - i0; d.c0 = d0;
    d.nA = (int32_t)(i1 - i0); d.nB = (int32_t)((d1 - i1) - (d0 - i0));
    d.first = 1;
    desc[k] = d;
}

// ---------------------------------------------------------------------------
// Steps 3-4 without the planning pass: one CTA per subproblem (used by the
// allocation-free entry point, whose scratch holds only the cross ranks)
// ---------------------------------------------------------------------------

template <typename K>
struct MergeArgs {
    const K* A; const uint32_t* Av; int64_t n;
    const K* B; const uint32_t* Bv; int64_t m;
    K* C; uint32_t* Cv;
    int64_t p;
    const int64_t* xbar; const int64_t* ybar;
    int32_t* status;
    int capA, capB;
    TileLayout lay;
};

template <typename K>
__global__ void __launch_bounds__(kMaxThreads)
tile_merge_kernel(const MergeArgs<K> g) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, T = blockDim.x;
    const int64_t item = blockIdx.x;
    const bool a_side = item < g.p;
    const int64_t pe = a_side ? item : item - g.p;

    int64_t a0, a1, b0, b1;
    auto xbar = [&](int64_t i) { return __ldg(g.xbar + i); };
    auto ybar = [&](int64_t j) { return __ldg(g.ybar + j); };
    subproblem_of<int64_t>(a_side, pe, g.n, g.m, g.p, xbar, ybar, a0, a1, b0, b1);
    const int64_t nA64 = a1 - a0, nB64 = b1 - b0;
    if (nA64 < 0 || nB64 < 0 || nA64 > g.capA || nB64 > g.capB) {
        if (tid == 0) set_status(g.status, TM_ERR_BOUNDS);
        return;
    }
    const int nA = (int)nA64, nB = (int)nB64;
    if (nA + nB == 0) return;

    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    uint8_t* rkA = smem + g.lay.off_kA; uint8_t* rvA = smem + g.lay.off_vA;
    uint8_t* rkB = smem + g.lay.off_kB; uint8_t* rvB = smem + g.lay.off_vB;
    uint8_t* rkC = smem + g.lay.off_kC; uint8_t* rvC = smem + g.lay.off_vC;

    const StageWin wkA = stage_window(g.A, g.n, a0, a1, sizeof(K));
    const StageWin wvA = stage_window(g.Av, g.n, a0, a1, 4);
    const StageWin wkB = stage_window(g.B, g.m, b0, b1, sizeof(K));
    const StageWin wvB = stage_window(g.Bv, g.m, b0, b1, 4);

    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fence_proxy_async_smem();
        uint32_t tx = wkA.bulk_bytes() + wvA.bulk_bytes() + wkB.bulk_bytes() + wvB.bulk_bytes();
        mbar_arrive_expect_tx(bar, tx);
        stage_issue(rkA, wkA, bar);
        stage_issue(rvA, wvA, bar);
        stage_issue(rkB, wkB, bar);
        stage_issue(rvB, wvB, bar);
    }
    stage_edges<K>(rkA, wkA, tid, T);
    stage_edges<uint32_t>(rvA, wvA, tid, T);
    stage_edges<K>(rkB, wkB, tid, T);
    stage_edges<uint32_t>(rvB, wvB, tid, T);
    __syncthreads();                                   // barrier initialised before anyone waits
    bool ok = mbar_wait_bounded(bar, 0, kWaitLimitNs);
    if (!__syncthreads_and(ok)) {
        if (tid == 0) set_status(g.status, TM_ERR_TIMEOUT);
        mbar_wait_bounded(bar, 0, kWaitLimitNs);       // let copies in flight land before exit
        return;
    }

    TileView<K> v;
    v.kA = reinterpret_cast<K*>(rkA) + wkA.head;
    v.vA = reinterpret_cast<uint32_t*>(rvA) + wvA.head;
    v.kB = reinterpret_cast<K*>(rkB) + wkB.head;
    v.vB = reinterpret_cast<uint32_t*>(rvB) + wvB.head;
    const OutWin ok_ = out_window(g.C, a0 + b0, nA + nB, sizeof(K));
    const OutWin ov_ = out_window(g.Cv, a0 + b0, nA + nB, 4);
    v.kC = reinterpret_cast<K*>(rkC + ok_.mis);
    v.vC = reinterpret_cast<uint32_t*>(rvC + ov_.mis);
    v.xs = reinterpret_cast<int*>(smem + g.lay.off_split);
    v.ys = v.xs + (T + 1);

    tile_resplit_and_merge<K>(v, nA, nB);

    if (tid == 0) {
        out_issue(ok_, rkC);
        out_issue(ov_, rvC);
        bulk_commit();
    }
    out_edges<K>(ok_, rkC, tid, T);
    out_edges<uint32_t>(ov_, rvC, tid, T);
    if (tid == 0) bulk_wait_read<0>();                 // smem must outlive the bulk store's reads
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

static int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }

int64_t choose_blocks(int64_t n, int64_t m, const tm_config* cfg) {
    if (cfg && cfg->p > 0) return cfg->p;
    int64_t tile = (cfg && cfg->tile > 0) ? cfg->tile : kDefaultTile;
    int64_t p = ceil_div64(n + m, tile);
    return p < 1 ? 1 : p;
}

int choose_threads(const tm_config* cfg) {
    return (cfg && cfg->threads > 0) ? cfg->threads : kDefaultThreads;
}

template <typename K>
static tm_status launch_tile_merge(const K* A, const uint32_t* Av, int64_t n,
                                   const K* B, const uint32_t* Bv, int64_t m,
                                   int64_t p, const int64_t* xbar, const int64_t* ybar,
                                   K* C, uint32_t* Cv, int32_t* status,
                                   const tm_config* cfg, cudaStream_t s) {
    MergeArgs<K> g;
    g.A = A; g.Av = Av; g.n = n; g.B = B; g.Bv = Bv; g.m = m; g.C = C; g.Cv = Cv;
    g.p = p; g.xbar = xbar; g.ybar = ybar; g.status = status;
    g.capA = (int)ceil_div64(n, p);
    g.capB = (int)ceil_div64(m, p);
    const int T = choose_threads(cfg);
    if (T < 64 || T > kMaxThreads || (T % 32) != 0) return TM_ERR_UNSUPPORTED;
    if (ceil_div64(n, p) + ceil_div64(m, p) > (int64_t)kMaxTileElems) return TM_ERR_UNSUPPORTED;
    g.lay = make_tile_layout(g.capA, g.capB, sizeof(K), T);
    if (g.lay.bytes > kMaxSmemBytes) return TM_ERR_UNSUPPORTED;
    if (!ensure_smem_limit(tile_merge_kernel<K>, g.lay.bytes)) return TM_ERR_UNSUPPORTED;
    if (2 * p > 0x7fffffffLL) return TM_ERR_UNSUPPORTED;
    tile_merge_kernel<K><<<(unsigned)(2 * p), T, g.lay.bytes, s>>>(g);
    return launch_status();
}

template <typename K>
static tm_status launch_cross_ranks(const K* A, int64_t n, const K* B, int64_t m, int64_t p,
                                    int64_t* xbar, int64_t* ybar, cudaStream_t s) {
    int64_t threads = 2 * p + 1;
    int64_t blocks = ceil_div64(threads, 256);
    if (blocks > 0x7fffffffLL) return TM_ERR_UNSUPPORTED;
    cross_rank_kernel<K><<<(unsigned)blocks, 256, 0, s>>>(A, n, B, m, p, xbar, ybar);
    return launch_status();
}

// ---------------------------------------------------------------------------
// Persistent tile engine launch
// ---------------------------------------------------------------------------

int log2_threads(const tm_config* cfg) {
    const int T = choose_threads(cfg);
    return T == 128 ? 7 : (T == 256 ? 8 : (T == 512 ? 9 : -1));
}

// Instantiated per key type in tm_engine_<type>.cu.
template <typename K>
tm_status launch_engine(const EngineArgs& a, const tm_config* cfg, cudaStream_t s);
extern template tm_status launch_engine<uint32_t>(const EngineArgs&, const tm_config*, cudaStream_t);
extern template tm_status launch_engine<int32_t>(const EngineArgs&, const tm_config*, cudaStream_t);
extern template tm_status launch_engine<uint64_t>(const EngineArgs&, const tm_config*, cudaStream_t);
extern template tm_status launch_engine<float>(const EngineArgs&, const tm_config*, cudaStream_t);
template <typename K>
tm_status launch_engine_fused(const EngineArgs& a, cudaStream_t s);
extern template tm_status launch_engine_fused<uint32_t>(const EngineArgs&, cudaStream_t);
extern template tm_status launch_engine_fused<int32_t>(const EngineArgs&, cudaStream_t);
extern template tm_status launch_engine_fused<uint64_t>(const EngineArgs&, cudaStream_t);
extern template tm_status launch_engine_fused<float>(const EngineArgs&, cudaStream_t);

template <typename K>
static tm_status merge_tiles_typed(const void* a_keys, const uint32_t* a_vals, int64_t n,
                                   const void* b_keys, const uint32_t* b_vals, int64_t m,
                                   const TileDesc* tiles, int64_t n_tiles, int cap,
                                   void* c_keys, uint32_t* c_vals, void* control,
                                   const tm_config* cfg, cudaStream_t s) {
    EngineArgs a{};
    a.desc = tiles; a.n_items = n_tiles; a.items_bound = n_tiles;
    a.status = reinterpret_cast<int32_t*>(control);
    a.queue = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(control) + 8);
    a.A = a_keys; a.Av = a_vals; a.lenA = n;
    a.B = b_keys; a.Bv = b_vals; a.lenB = m;
    a.C = c_keys; a.Cv = c_vals;
    a.vbytes = payload_size(cfg);
    a.cap = cap;
    return launch_engine<K>(a, cfg, s);
}

tm_status merge_tiles_dispatch(tm_key_type kt, const void* a_keys, const uint32_t* a_vals, int64_t n,
                               const void* b_keys, const uint32_t* b_vals, int64_t m,
                               const void* tiles, int64_t n_tiles, int cap,
                               void* c_keys, uint32_t* c_vals, void* control,
                               const tm_config* cfg, cudaStream_t s) {
    const TileDesc* t = static_cast<const TileDesc*>(tiles);
    switch (kt) {
        case TM_KEY_U32: return merge_tiles_typed<uint32_t>(a_keys, a_vals, n, b_keys, b_vals, m, t, n_tiles, cap, c_keys, c_vals, control, cfg, s);
        case TM_KEY_I32: return merge_tiles_typed<int32_t>(a_keys, a_vals, n, b_keys, b_vals, m, t, n_tiles, cap, c_keys, c_vals, control, cfg, s);
        case TM_KEY_U64: return merge_tiles_typed<uint64_t>(a_keys, a_vals, n, b_keys, b_vals, m, t, n_tiles, cap, c_keys, c_vals, control, cfg, s);
        case TM_KEY_F32: return merge_tiles_typed<float>(a_keys, a_vals, n, b_keys, b_vals, m, t, n_tiles, cap, c_keys, c_vals, control, cfg, s);
    }
    return TM_ERR_UNSUPPORTED;
}

static tm_status launch_plan_single(int64_t n, int64_t m, int64_t p, const int64_t* xbar, const int64_t* ybar,
                                    TileDesc* desc, cudaStream_t s) {
    int64_t blocks = (2 * p + 255) / 256;
    if (blocks > 0x7fffffffLL) return TM_ERR_UNSUPPORTED;
    plan_single_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, m, p, xbar, ybar, desc);
    return launch_status();
}

// Largest subproblem of the single merge: one A-block piece plus one B-block
// piece (Section 2: the ranges of cases (a)-(e) lie inside blocks).
static int64_t single_merge_cap(int64_t n, int64_t m, int64_t p) {
    return ceil_div64(n, p) + ceil_div64(m, p);
}

// Non-empty subproblems: one per non-empty block of either array.
static int64_t single_merge_tiles(int64_t n, int64_t m, int64_t p) {
    return (n < p ? n : p) + (m < p ? m : p);
}

// Workspace of tm_merge: [status int32 | queue u64 | grid-barrier count u32 | pad to 256] xbar ybar tiles
// [trace: kTraceSlots u64 per CTA, plus a header row, when cfg->trace].
struct MergeWs {
    int32_t* status; void* control; int64_t* xbar; int64_t* ybar; TileDesc* tiles; uint64_t* trace; size_t bytes;
};

constexpr int64_t kTraceMaxCtas = 4096;

static bool wants_trace(const tm_config* cfg) { return cfg && cfg->trace; }

static MergeWs merge_ws_layout(void* base, int64_t p, bool trace) {
    MergeWs w;
    uint8_t* b = static_cast<uint8_t*>(base);
    size_t o = kStatusBytes;
    w.status = reinterpret_cast<int32_t*>(b);
    w.control = b;
    w.xbar = reinterpret_cast<int64_t*>(b + o); o += align_up((size_t)(p + 1) * 8, 256);
    w.ybar = reinterpret_cast<int64_t*>(b + o); o += align_up((size_t)(p + 1) * 8, 256);
    w.tiles = reinterpret_cast<TileDesc*>(b + o); o += align_up((size_t)(2 * p) * sizeof(TileDesc), 256);
    w.trace = nullptr;
    if (trace) {
        w.trace = reinterpret_cast<uint64_t*>(b + o);
        o += align_up((size_t)(kTraceMaxCtas + 1) * kTraceSlots * 8, 256);
    }
    w.bytes = o;
    return w;
}

size_t merge_workspace_bytes(int64_t p, const tm_config* cfg) { return merge_ws_layout(nullptr, p, wants_trace(cfg)).bytes; }

// The fused single launch applies to small merges with the default in-CTA
// settings (it has one configuration: 128 consumer threads, diagonal split,
// 4 stages) on a device that supports cooperative launches.
constexpr int64_t kFusedMaxBlocks = 16384;
constexpr int64_t kFusedMaxCap = 17 * 128;

static bool fused_applies(int64_t p, int64_t cap, const tm_config* cfg) {
    if (p > kFusedMaxBlocks || cap > kFusedMaxCap) return false;
    if (sm_count() * 8 > kTraceMaxCtas) return false;  // more CTAs than a trace holds
    if (cfg && (cfg->unfused || cfg->partition || (cfg->threads && cfg->threads != 128) || cfg->stages || cfg->grid ||
                (cfg->split && cfg->split != TM_SPLIT_DIAGONAL) || cfg->wait_ms || cfg->test_drop_tile))
        return false;
    int dev = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    return cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop;
}

// Merges beyond the fused launch's range, called with the default
// configuration, get the shape measured best for their layout (n = m = 2^28
// int32 keys): keys only take 8192-element tiles and 256 consumer threads
// (without payload regions such stages still fit two CTAs per SM, and the
// longer per-thread runs spread the co-rank search and the per-tile work:
// uniform keys 0.90 -> 0.83 ms, keys in [0, 1024) 0.69 -> 0.67 ms); 8-byte
// payloads take 256 consumer threads (uniform keys 2.07 -> 1.99 ms).  The
// block count p follows the tile, never above the default one, so the
// default workspace size still covers it.
constexpr int kKeysOnlyTile = 8192;
constexpr int kWideThreads = 256;

static bool layout_config(const void* a_vals, const void* b_vals, int64_t n, int64_t m, const tm_config* cfg,
                          tm_config* out) {
    const bool keys_only = a_vals == nullptr && b_vals == nullptr;
    if (!keys_only && payload_size(cfg) != 8) return false;
    if (cfg) {                                         // nothing set but fields that do not apply here
        tm_config d{};
        d.payload_bytes = cfg->payload_bytes;
        d.merge_ways = cfg->merge_ways;
        if (std::memcmp(&d, cfg, sizeof(tm_config)) != 0) return false;
    }
    if (choose_blocks(n, m, cfg) <= kFusedMaxBlocks) return false;
    *out = cfg ? *cfg : tm_config{};
    if (keys_only) out->tile = kKeysOnlyTile;
    out->threads = kWideThreads;
    return true;
}

template <typename K>
static tm_status merge_typed(tm_key_type kt, const void* a_keys, const uint32_t* a_vals, int64_t n,
                             const void* b_keys, const uint32_t* b_vals, int64_t m,
                             void* c_keys, uint32_t* c_vals, void* ws, int64_t p,
                             const tm_config* cfg, cudaStream_t s) {
    MergeWs w = merge_ws_layout(ws, p, wants_trace(cfg));
    // status word, work-queue counter, grid-barrier count
    if (cudaError_t e = cudaMemsetAsync(w.control, 0, 32, s); e != cudaSuccess) return cuda_failed(e);
    if (w.trace) {                                     // no trace until a fused launch writes one
        if (cudaError_t e = cudaMemsetAsync(w.trace, 0, 8, s); e != cudaSuccess) return cuda_failed(e);
    }
    if (n + m == 0) return TM_OK;
    if (log2_threads(cfg) < 0) return TM_ERR_UNSUPPORTED;
    const int64_t cap = single_merge_cap(n, m, p);
    if (cap > kMaxTileElems) return TM_ERR_UNSUPPORTED;
    const K* A = static_cast<const K*>(a_keys);
    const K* B = static_cast<const K*>(b_keys);
    if (cfg && cfg->partition == TM_PARTITION_DIAGONALS) {   // ablation: equal output ranges
        if (cfg->p > 0) return TM_ERR_UNSUPPORTED;            // the cut count follows the tile
        const int64_t tile = (cfg->tile > 0) ? cfg->tile : kDefaultTile;
        const int64_t cuts = ceil_div64(n + m, tile);          // == p, the workspace's sizing
        if (tile > kMaxTileElems || cuts + 1 > 0x7fffffffLL * 256) return TM_ERR_UNSUPPORTED;
        diagonal_corank_kernel<K><<<(unsigned)((cuts + 1 + 255) / 256), 256, 0, s>>>(A, n, B, m, tile, cuts,
                                                                                    w.xbar);
        diagonal_plan_kernel<<<(unsigned)((cuts + 255) / 256), 256, 0, s>>>(n, m, tile, cuts, w.xbar, w.tiles);
        if (const cudaError_t e = cudaGetLastError(); e != cudaSuccess) return cuda_failed(e);
        return merge_tiles_dispatch(kt, a_keys, a_vals, n, b_keys, b_vals, m, w.tiles, cuts, (int)tile,
                                    c_keys, c_vals, w.control, cfg, s);
    } else if (cfg && cfg->partition != TM_PARTITION_BLOCKS) {
        return TM_ERR_UNSUPPORTED;
    }
    if (fused_applies(p, cap, cfg)) {
        EngineArgs a{};
        a.desc = w.tiles;
        a.n_items = single_merge_tiles(n, m, p); a.items_bound = a.n_items;
        a.status = w.status;
        a.queue = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(w.control) + 8);
        a.A = a_keys; a.Av = a_vals; a.lenA = n;
        a.B = b_keys; a.Bv = b_vals; a.lenB = m;
        a.C = c_keys; a.Cv = c_vals;
        a.vbytes = payload_size(cfg);
        a.cap = (int)cap;
        a.fx = w.xbar; a.fy = w.ybar; a.fp = p;
        a.fbA = Blocks32((uint32_t)n, (uint32_t)p);     // n, m <= kFusedMaxBlocks * kFusedMaxCap < 2^31
        a.fbB = Blocks32((uint32_t)m, (uint32_t)p);
        a.gbar = reinterpret_cast<unsigned int*>(static_cast<uint8_t*>(w.control) + 16);
        a.trace = w.trace;
        const tm_status st = launch_engine_fused<K>(a, s);
        if (st != TM_ERR_UNSUPPORTED) return st;       // else: the separate launches below
    }
    tm_status st = launch_cross_ranks<K>(A, n, B, m, p, w.xbar, w.ybar, s);
    if (st != TM_OK) return st;
    st = launch_plan_single(n, m, p, w.xbar, w.ybar, w.tiles, s);
    if (st != TM_OK) return st;
    return merge_tiles_dispatch(kt, a_keys, a_vals, n, b_keys, b_vals, m, w.tiles, single_merge_tiles(n, m, p),
                                (int)cap, c_keys, c_vals, w.control, cfg, s);
}

}  // namespace pmerge

using namespace pmerge;

extern "C" {

const char* tm_status_str(tm_status s) {
    switch (s) {
        case TM_OK: return "ok";
        case TM_ERR_INVALID: return "invalid argument";
        case TM_ERR_UNSUPPORTED: return "unsupported key type or configuration";
        case TM_ERR_WORKSPACE: return "workspace missing or too small";
        case TM_ERR_CUDA: return "CUDA error";
        case TM_ERR_TIMEOUT: return "device wait timed out";
        case TM_ERR_BOUNDS: return "subproblem exceeded its staging capacity";
    }
    return "unknown status";
}

int tm_version(void) { return kVersion; }

const char* tm_last_cuda_error(void) { return cudaGetErrorName(last_cuda_error()); }

tm_status tm_read_status(const void* status, tm_stream_t stream) {
    if (!status) return TM_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (const cudaError_t e = cudaStreamSynchronize(s); e != cudaSuccess) return cuda_failed(e);
    int32_t h = 0;
    if (const cudaError_t e = cudaMemcpy(&h, status, sizeof(h), cudaMemcpyDeviceToHost); e != cudaSuccess)
        return cuda_failed(e);
    return static_cast<tm_status>(h);
}

int64_t tm_merge_blocks(int64_t n, int64_t m, const tm_config* cfg) {
    if (n < 0 || m < 0) return -1;
    return choose_blocks(n, m, cfg);
}

size_t tm_merge_workspace_size(int64_t n, int64_t m, const tm_config* cfg) {
    if (n < 0 || m < 0) return 0;
    return merge_workspace_bytes(choose_blocks(n, m, cfg), cfg);
}

}  // extern "C"

namespace {
// The stamps of the last traced fused launch on `workspace`: grid CTAs of
// kTraceSlots words each, after synchronising `stream`.
tm_status read_trace(const void* workspace, int64_t n, int64_t m, const tm_config* cfg, tm_stream_t stream,
                     std::vector<uint64_t>& t, uint64_t& grid) {
    if (n < 0 || m < 0 || !wants_trace(cfg) || !aligned(workspace, 256)) return TM_ERR_INVALID;
    const MergeWs w = merge_ws_layout(const_cast<void*>(workspace), choose_blocks(n, m, cfg), true);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (const cudaError_t e = cudaStreamSynchronize(s); e != cudaSuccess) return cuda_failed(e);
    grid = 0;
    if (const cudaError_t e = cudaMemcpy(&grid, w.trace, 8, cudaMemcpyDeviceToHost); e != cudaSuccess)
        return cuda_failed(e);
    if (grid == 0 || grid > (uint64_t)kTraceMaxCtas) return TM_ERR_INVALID;
    t.assign((size_t)grid * kTraceSlots, 0);
    if (const cudaError_t e = cudaMemcpy(t.data(), w.trace + kTraceSlots, t.size() * 8, cudaMemcpyDeviceToHost);
        e != cudaSuccess)
        return cuda_failed(e);
    return TM_OK;
}
}  // namespace

extern "C" {

tm_status tm_merge_phase_times(const void* workspace, int64_t n, int64_t m, const tm_config* cfg,
                               double* us_out, tm_stream_t stream) {
    if (!us_out) return TM_ERR_INVALID;
    std::vector<uint64_t> t;
    uint64_t grid = 0;
    if (const tm_status st = read_trace(workspace, n, m, cfg, stream, t, grid); st != TM_OK) return st;
    // phase ends: the last CTA to reach each stamp; start: the first entry
    uint64_t start = UINT64_MAX, end[6] = {0, 0, 0, 0, 0, 0};
    for (uint64_t c = 0; c < grid; ++c) {
        const uint64_t* r = &t[(size_t)c * kTraceSlots];
        start = std::min(start, r[0]);
        for (int k = 1; k <= 5; ++k) end[k] = std::max(end[k], r[k]);
    }
    end[0] = start;
    for (int k = 1; k <= 5; ++k) end[k] = std::max(end[k], end[k - 1]);   // a phase never ends before the last
    for (int k = 0; k < 5; ++k) us_out[k] = (double)(end[k + 1] - end[k]) * 1e-3;
    us_out[5] = (double)(end[5] - start) * 1e-3;
    return TM_OK;
}

tm_status tm_merge_trace(const void* workspace, int64_t n, int64_t m, const tm_config* cfg, uint64_t* out,
                         int64_t capacity, int64_t* ctas, tm_stream_t stream) {
    if (!ctas || capacity < 0 || (capacity > 0 && !out)) return TM_ERR_INVALID;   // capacity 0: the count only
    std::vector<uint64_t> t;
    uint64_t grid = 0;
    if (const tm_status st = read_trace(workspace, n, m, cfg, stream, t, grid); st != TM_OK) return st;
    *ctas = (int64_t)grid;
    if ((uint64_t)capacity < t.size()) return TM_ERR_INVALID;
    std::copy(t.begin(), t.end(), out);
    return TM_OK;
}

tm_status tm_merge(tm_key_type kt,
                   const void* a_keys, const uint32_t* a_vals, int64_t n,
                   const void* b_keys, const uint32_t* b_vals, int64_t m,
                   void* c_keys, uint32_t* c_vals,
                   void* workspace, size_t workspace_bytes,
                   const tm_config* cfg, tm_stream_t stream) {
    if (n < 0 || m < 0) return TM_ERR_INVALID;
    if (kt < TM_KEY_U32 || kt > TM_KEY_F32 || payload_size(cfg) < 0) return TM_ERR_UNSUPPORTED;
    const size_t E = key_size(kt);
    if ((n > 0 && !aligned(a_keys, E)) || (m > 0 && !aligned(b_keys, E)) || (n + m > 0 && !aligned(c_keys, E)) ||
        !payloads_ok(n, a_vals, m, b_vals, c_vals, payload_size(cfg)))
        return TM_ERR_INVALID;
    int64_t p = choose_blocks(n, m, cfg);
    if (!workspace || !aligned(workspace, 256) || workspace_bytes < merge_workspace_bytes(p, cfg))
        return TM_ERR_WORKSPACE;
    tm_config shaped;
    if (layout_config(a_vals, b_vals, n, m, cfg, &shaped)) {   // p no larger: the workspace covers it
        cfg = &shaped;
        p = choose_blocks(n, m, cfg);
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (kt) {
        case TM_KEY_U32: return merge_typed<uint32_t>(kt, a_keys, a_vals, n, b_keys, b_vals, m, c_keys, c_vals, workspace, p, cfg, s);
        case TM_KEY_I32: return merge_typed<int32_t>(kt, a_keys, a_vals, n, b_keys, b_vals, m, c_keys, c_vals, workspace, p, cfg, s);
        case TM_KEY_U64: return merge_typed<uint64_t>(kt, a_keys, a_vals, n, b_keys, b_vals, m, c_keys, c_vals, workspace, p, cfg, s);
        case TM_KEY_F32: return merge_typed<float>(kt, a_keys, a_vals, n, b_keys, b_vals, m, c_keys, c_vals, workspace, p, cfg, s);
    }
    return TM_ERR_UNSUPPORTED;
}

tm_status tm_cross_ranks(tm_key_type kt, const void* a_keys, int64_t n,
                         const void* b_keys, int64_t m, int64_t p,
                         int64_t* xbar, int64_t* ybar, tm_stream_t stream) {
    if (n < 0 || m < 0 || p < 1 || !xbar || !ybar) return TM_ERR_INVALID;
    if (kt < TM_KEY_U32 || kt > TM_KEY_F32) return TM_ERR_UNSUPPORTED;
    const size_t E = key_size(kt);
    if ((n > 0 && !aligned(a_keys, E)) || (m > 0 && !aligned(b_keys, E)) ||
        !aligned(xbar, 8) || !aligned(ybar, 8))
        return TM_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (kt) {
        case TM_KEY_U32: return launch_cross_ranks<uint32_t>((const uint32_t*)a_keys, n, (const uint32_t*)b_keys, m, p, xbar, ybar, s);
        case TM_KEY_I32: return launch_cross_ranks<int32_t>((const int32_t*)a_keys, n, (const int32_t*)b_keys, m, p, xbar, ybar, s);
        case TM_KEY_U64: return launch_cross_ranks<uint64_t>((const uint64_t*)a_keys, n, (const uint64_t*)b_keys, m, p, xbar, ybar, s);
        case TM_KEY_F32: return launch_cross_ranks<float>((const float*)a_keys, n, (const float*)b_keys, m, p, xbar, ybar, s);
    }
    return TM_ERR_UNSUPPORTED;
}

size_t tm_tile_record_bytes(void) { return sizeof(TileDesc); }

int32_t tm_merge_tile_cap(int64_t n, int64_t m, int64_t p) {
    if (n < 0 || m < 0 || p < 1) return -1;
    int64_t c = single_merge_cap(n, m, p);
    return c > 0x7fffffff ? -1 : (int32_t)c;
}

int64_t tm_plan_tile_count(int64_t n, int64_t m, int64_t p) {
    if (n < 0 || m < 0 || p < 1) return -1;
    return single_merge_tiles(n, m, p);
}

tm_status tm_plan_subproblems(int64_t n, int64_t m, int64_t p, const int64_t* xbar, const int64_t* ybar,
                              void* tiles, const tm_config* cfg, tm_stream_t stream) {
    (void)cfg;
    if (n < 0 || m < 0 || p < 1 || !aligned(xbar, 8) || !aligned(ybar, 8) || !aligned(tiles, 16))
        return TM_ERR_INVALID;
    return launch_plan_single(n, m, p, xbar, ybar, static_cast<TileDesc*>(tiles),
                              reinterpret_cast<cudaStream_t>(stream));
}

tm_status tm_merge_tiles(tm_key_type kt,
                         const void* a_keys, const uint32_t* a_vals, int64_t n,
                         const void* b_keys, const uint32_t* b_vals, int64_t m,
                         const void* tiles, int64_t n_tiles, int32_t cap,
                         void* c_keys, uint32_t* c_vals, void* control,
                         const tm_config* cfg, tm_stream_t stream) {
    if (n < 0 || m < 0 || n_tiles < 0 || cap < 1 || !aligned(control, 256)) return TM_ERR_INVALID;
    if (kt < TM_KEY_U32 || kt > TM_KEY_F32 || payload_size(cfg) < 0) return TM_ERR_UNSUPPORTED;
    const size_t E = key_size(kt);
    if ((n > 0 && !aligned(a_keys, E)) || (m > 0 && !aligned(b_keys, E)) || (n + m > 0 && !aligned(c_keys, E)) ||
        !payloads_ok(n, a_vals, m, b_vals, c_vals, payload_size(cfg)) || (n_tiles > 0 && !aligned(tiles, 16)))
        return TM_ERR_INVALID;
    if (n_tiles == 0 || n + m == 0) return TM_OK;
    return merge_tiles_dispatch(kt, a_keys, a_vals, n, b_keys, b_vals, m, tiles, n_tiles, cap,
                                c_keys, c_vals, control, cfg, reinterpret_cast<cudaStream_t>(stream));
}

tm_status tm_subproblems(int64_t n, int64_t m, int64_t p, const int64_t* xbar,
                         const int64_t* ybar, int64_t* table, tm_stream_t stream) {
    if (n < 0 || m < 0 || p < 1 || !aligned(xbar, 8) || !aligned(ybar, 8) || !aligned(table, 8))
        return TM_ERR_INVALID;
    int64_t blocks = (2 * p + 255) / 256;
    if (blocks > 0x7fffffffLL) return TM_ERR_UNSUPPORTED;
    subproblem_table_kernel<<<(unsigned)blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        n, m, p, xbar, ybar, table);
    return launch_status();
}

tm_status tm_rank_search(tm_key_type kt, int kind, const void* q, int64_t count,
                         const void* x_keys, int64_t len, int64_t* out, tm_stream_t stream) {
    if (count < 0 || len < 0 || (kind != 0 && kind != 1)) return TM_ERR_INVALID;
    if (kt < TM_KEY_U32 || kt > TM_KEY_F32) return TM_ERR_UNSUPPORTED;
    if (count == 0) return TM_OK;
    const size_t E = key_size(kt);
    if (!aligned(q, E) || (len > 0 && !aligned(x_keys, E)) || !aligned(out, 8)) return TM_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int64_t blocks = (count + 255) / 256;
    if (blocks > 0x7fffffffLL) return TM_ERR_UNSUPPORTED;
    switch (kt) {
        case TM_KEY_U32: rank_search_kernel<uint32_t><<<(unsigned)blocks, 256, 0, s>>>((const uint32_t*)q, count, (const uint32_t*)x_keys, len, kind, out); break;
        case TM_KEY_I32: rank_search_kernel<int32_t><<<(unsigned)blocks, 256, 0, s>>>((const int32_t*)q, count, (const int32_t*)x_keys, len, kind, out); break;
        case TM_KEY_U64: rank_search_kernel<uint64_t><<<(unsigned)blocks, 256, 0, s>>>((const uint64_t*)q, count, (const uint64_t*)x_keys, len, kind, out); break;
        case TM_KEY_F32: rank_search_kernel<float><<<(unsigned)blocks, 256, 0, s>>>((const float*)q, count, (const float*)x_keys, len, kind, out); break;
    }
    return launch_status();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Merge without allocation: the cross ranks live in a file-scope device array
// ---------------------------------------------------------------------------
// For callers that can neither allocate device memory nor supply a workspace.
// The array is part of this module, so every GPU that loads the library
// holds it (4 MiB) until the process exits.

namespace pmerge {

constexpr int64_t kNoAllocMaxBlocks = 262143;            // p + 1 <= 262144 per side

static __device__ __align__(256) int64_t g_noalloc_ranks[2 * (kNoAllocMaxBlocks + 1)];

// The calling thread's current CUDA context, through the driver's
// cuCtxGetCurrent (found once via the runtime, so the library does not link
// libcuda); nullptr if it cannot be found.
static void* current_context() {
    using CtxGetCurrent = int (*)(void**);            // CUresult cuCtxGetCurrent(CUcontext*)
    static CtxGetCurrent fn = []() -> CtxGetCurrent {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<CtxGetCurrent>(f);
    }();
    void* ctx = nullptr;
    if (!fn || fn(&ctx) != 0) return nullptr;
    return ctx;
}

// Device address of g_noalloc_ranks for the current device and context,
// looked up once per (device, context) with that device current: the
// host-side name of a __device__ array is not a device address, and a
// context created after cudaDeviceReset holds the array at a new address.
static int64_t* noalloc_ranks_ptr() {
    static std::mutex mu;
    static void* ctx_of[64] = {nullptr};
    static int64_t* addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    void* ctx = current_context();                    // nullptr before the runtime's first use
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev] || ctx == nullptr || ctx != ctx_of[dev]) {
        void* p = nullptr;
        if (const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_ranks); e != cudaSuccess) {
            record_cuda_error(e);
            return nullptr;
        }
        addr[dev] = static_cast<int64_t*>(p);
        ctx_of[dev] = current_context();              // the lookup made the device's context current
    }
    return addr[dev];
}

template <typename K>
static tm_status merge_noalloc_typed(const void* a_keys, const uint32_t* a_vals, int64_t n,
                                     const void* b_keys, const uint32_t* b_vals, int64_t m,
                                     void* c_keys, uint32_t* c_vals, int32_t* status,
                                     int64_t p, const tm_config* cfg, cudaStream_t s) {
    int64_t* ranks = noalloc_ranks_ptr();
    if (!ranks) return TM_ERR_CUDA;
    int64_t* xbar = ranks;
    int64_t* ybar = ranks + (kNoAllocMaxBlocks + 1);
    if (status) {
        if (const cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), s); e != cudaSuccess)
            return cuda_failed(e);
    }
    if (n + m == 0) return TM_OK;
    const K* A = static_cast<const K*>(a_keys);
    const K* B = static_cast<const K*>(b_keys);
    tm_status st = launch_cross_ranks<K>(A, n, B, m, p, xbar, ybar, s);
    if (st != TM_OK) return st;
    return launch_tile_merge<K>(A, a_vals, n, B, b_vals, m, p, xbar, ybar,
                                static_cast<K*>(c_keys), c_vals, status, cfg, s);
}

}  // namespace pmerge

extern "C" tm_status tm_merge_noalloc(tm_key_type kt,
                                      const void* a_keys, const uint32_t* a_vals, int64_t n,
                                      const void* b_keys, const uint32_t* b_vals, int64_t m,
                                      void* c_keys, uint32_t* c_vals, int32_t* status,
                                      const tm_config* cfg, tm_stream_t stream) {
    using namespace pmerge;
    if (n < 0 || m < 0) return TM_ERR_INVALID;
    if (kt < TM_KEY_U32 || kt > TM_KEY_F32) return TM_ERR_UNSUPPORTED;
    const size_t E = key_size(kt);
    if ((n > 0 && (!aligned(a_keys, E) || !aligned(a_vals, 4))) ||
        (m > 0 && (!aligned(b_keys, E) || !aligned(b_vals, 4))) ||
        (n + m > 0 && (!aligned(c_keys, E) || !aligned(c_vals, 4))) ||
        (status && !aligned(status, 4)))
        return c_vals == nullptr && a_vals == nullptr && b_vals == nullptr ? TM_ERR_UNSUPPORTED : TM_ERR_INVALID;
    // one method only: the paper's blocks, one CTA per subproblem, 128, 256
    // or 512 threads (split, stages, grid and unfused do not apply)
    if (cfg && (cfg->partition != TM_PARTITION_BLOCKS || (cfg->threads && log2_threads(cfg) < 0) ||
                payload_size(cfg) != 4))
        return TM_ERR_UNSUPPORTED;
    const int64_t p = choose_blocks(n, m, cfg);
    if (p > kNoAllocMaxBlocks) return TM_ERR_WORKSPACE;   // beyond the built-in array
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (kt) {
        case TM_KEY_U32: return merge_noalloc_typed<uint32_t>(a_keys, a_vals, n, b_keys, b_vals, m, c_keys, c_vals, status, p, cfg, s);
        case TM_KEY_I32: return merge_noalloc_typed<int32_t>(a_keys, a_vals, n, b_keys, b_vals, m, c_keys, c_vals, status, p, cfg, s);
        case TM_KEY_U64: return merge_noalloc_typed<uint64_t>(a_keys, a_vals, n, b_keys, b_vals, m, c_keys, c_vals, status, p, cfg, s);
        case TM_KEY_F32: return merge_noalloc_typed<float>(a_keys, a_vals, n, b_keys, b_vals, m, c_keys, c_vals, status, p, cfg, s);
    }
    return TM_ERR_UNSUPPORTED;
}
