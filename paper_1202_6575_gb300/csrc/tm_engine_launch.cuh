// Host-side launch of the persistent tile engine: picks the pipeline depth
// (input stages, output buffers) and the grid from the tile capacity, the
// key size and the device's shared memory.  Instantiated once per key type
// in tm_engine_<type>.cu so the key types compile in parallel.
#pragma once

#include "tm_engine.cuh"
#include "tm_host.h"

namespace pmerge {

// Resident CTAs of `bytes` dynamic shared memory on one SM (1 KB reserved per CTA).
inline int ctas_by_smem(uint32_t bytes) {
    int dev = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
        return 0;
    return per_sm / (int)(bytes + 1024);
}

// Diagonal split: the consumers hold VT * T outputs, usually more than the
// largest record.  Staging that many lets two neighbouring records of about
// half a tile pack into one tile far more often (their sum exceeds the
// largest single record about half the time), as long as the larger stages
// keep the same number of CTAs per SM.
template <typename K, int LOG_T, int S_IN, int S_OUT, int VT>
int packing_cap(int cap, int vsize) {
    const int full = VT << LOG_T;
    if (cap >= full) return cap;
    const uint32_t now = make_engine_layout(cap, sizeof(K), vsize, 1 << LOG_T, S_IN, S_OUT).total;
    const uint32_t more = make_engine_layout(full, sizeof(K), vsize, 1 << LOG_T, S_IN, S_OUT).total;
    const int c0 = ctas_by_smem(now);
    return (c0 > 0 && ctas_by_smem(more) >= c0) ? full : cap;
}

// Consumer groups per CTA (each merges every NG-th tile on S_IN / NG stages
// of its own).  Streaming launches keep one: a group holds two stages (the
// tile it merges and the one whose store is still reading), so with two
// groups on four stages the producer has none left to load ahead into
// (measured: keys-only merge 0.90 -> 1.54 ms).  The fused small merge
// stages all of a CTA's 2-4 tiles at once and takes two (24.7 -> 22.6 us).
constexpr int kConsumerGroups = 1;
constexpr int kFusedConsumerGroups = 2;

// Payload bytes a launch stages per element: 0 for a keys-only merge.
inline int staged_vsize(const EngineArgs& a) { return a.Cv ? a.vbytes : 0; }

template <typename K, typename V, int LOG_T, int S_IN, int S_OUT, int SPLIT, int VT>
tm_status launch_engine_s(const EngineArgs& a_in, const tm_config* cfg, cudaStream_t s) {
    EngineArgs a = a_in;
    const int vs = staged_vsize(a);
    if constexpr (SPLIT == kSplitDiagonal) a.cap = packing_cap<K, LOG_T, S_IN, S_OUT, VT>(a.cap, vs);
    a.lay = make_engine_layout(a.cap, sizeof(K), vs, 1 << LOG_T, S_IN, S_OUT);
    a.wait_ns = (cfg && cfg->wait_ms > 0) ? (uint64_t)cfg->wait_ms * 1000000ull : kWaitLimitNs;
    a.drop_fill = (cfg && cfg->test_drop_tile > 0) ? cfg->test_drop_tile - 1 : -1;
    constexpr int NG = (SPLIT == kSplitDiagonal && S_IN == 2 * kConsumerGroups) ? kConsumerGroups : 1;
    auto kern = merge_engine_kernel<K, V, LOG_T, S_IN, S_OUT, SPLIT, VT, false, NG>;
    if (!ensure_smem_limit(kern, a.lay.total)) return TM_ERR_UNSUPPORTED;
    const int block = (1 << LOG_T) * NG + 32;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, a.lay.total) != cudaSuccess || per_sm < 1)
        return TM_ERR_UNSUPPORTED;
    int64_t grid = (int64_t)per_sm * sm_count();
    if (cfg && cfg->grid > 0) grid = cfg->grid;
    // n_items may live on the device (batched form); then size by its bound
    const int64_t items = a.n_items >= 0 ? a.n_items : a.items_bound;
    int64_t g = items / (grid * 8);
    a.grab = (int)(g < 1 ? 1 : (g > 16 ? 16 : g));
    int64_t need = (items + a.grab - 1) / a.grab;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    if (cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s) != cudaSuccess) return TM_ERR_CUDA;
    kern<<<(unsigned)grid, block, a.lay.total, s>>>(a);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TM_OK : cuda_failed(e);
}

// Paper's rule inside the CTA, with separate output buffers.  cfg->stages:
// 4, 2 or 1 input stages; 0 picks 2 (1 when two do not fit).
template <typename K, typename V, int LOG_T>
tm_status launch_blocks(const EngineArgs& a, const tm_config* cfg, cudaStream_t s) {
    const int want = (cfg && cfg->stages > 0) ? cfg->stages : 0;
    switch (want) {
        case 4: return launch_engine_s<K, V, LOG_T, 4, 2, kSplitBlocks, 1>(a, cfg, s);
        case 2: return launch_engine_s<K, V, LOG_T, 2, 2, kSplitBlocks, 1>(a, cfg, s);
        case 1: return launch_engine_s<K, V, LOG_T, 1, 1, kSplitBlocks, 1>(a, cfg, s);
        case 0: break;
        default: return TM_ERR_UNSUPPORTED;
    }
    if (make_engine_layout(a.cap, sizeof(K), staged_vsize(a), 1 << LOG_T, 2, 2).total <= device_smem_limit())
        return launch_engine_s<K, V, LOG_T, 2, 2, kSplitBlocks, 1>(a, cfg, s);
    return launch_engine_s<K, V, LOG_T, 1, 1, kSplitBlocks, 1>(a, cfg, s);
}

// Equal output runs of VT elements per thread, output written back into the
// consumed stage (no output buffers).  A stage stays busy until the next
// tile is merged, so at least 2 stages; cfg->stages 2, 3 or 4; default 4
// when two such CTAs share an SM, else 3, else 2.
template <typename K, typename V, int LOG_T, int VT>
tm_status launch_diagonal_vt(const EngineArgs& a, const tm_config* cfg, cudaStream_t s) {
    const int want = (cfg && cfg->stages > 0) ? cfg->stages : 0;
    switch (want) {
        case 4: return launch_engine_s<K, V, LOG_T, 4, 0, kSplitDiagonal, VT>(a, cfg, s);
        case 3: return launch_engine_s<K, V, LOG_T, 3, 0, kSplitDiagonal, VT>(a, cfg, s);
        case 2: return launch_engine_s<K, V, LOG_T, 2, 0, kSplitDiagonal, VT>(a, cfg, s);
        case 0: break;
        default: return TM_ERR_UNSUPPORTED;
    }
    const uint32_t lim = device_smem_limit();
    const uint32_t half = lim / 2 > 2048 ? lim / 2 - 2048 : 0;
    const int vs = staged_vsize(a);
    if (make_engine_layout(a.cap, sizeof(K), vs, 1 << LOG_T, 4, 0).total <= half)
        return launch_engine_s<K, V, LOG_T, 4, 0, kSplitDiagonal, VT>(a, cfg, s);
    if (make_engine_layout(a.cap, sizeof(K), vs, 1 << LOG_T, 3, 0).total <= lim)
        return launch_engine_s<K, V, LOG_T, 3, 0, kSplitDiagonal, VT>(a, cfg, s);
    return launch_engine_s<K, V, LOG_T, 2, 0, kSplitDiagonal, VT>(a, cfg, s);
}

// Smallest odd run length VT in {9, 17, 33} with T * VT >= cap.
template <typename K, typename V, int LOG_T>
tm_status launch_diagonal(const EngineArgs& a, const tm_config* cfg, cudaStream_t s) {
    const int T = 1 << LOG_T;
    if (a.cap <= 9 * T) return launch_diagonal_vt<K, V, LOG_T, 9>(a, cfg, s);
    if (a.cap <= 17 * T) return launch_diagonal_vt<K, V, LOG_T, 17>(a, cfg, s);
    if (a.cap <= 33 * T) return launch_diagonal_vt<K, V, LOG_T, 33>(a, cfg, s);
    return TM_ERR_UNSUPPORTED;
}

// Fused single merge: one cooperative launch (every CTA resident, so the
// grid barrier after the searches cannot wait on an unscheduled CTA),
// 128 consumer threads, diagonal split, 4 input stages.  The work queue and
// the barrier words must be zero (the caller clears the control block).
template <typename K, typename V, int VT>
tm_status launch_fused_vt(const EngineArgs& a_in, cudaStream_t s) {
    constexpr int LOG_T = 7;
    EngineArgs a = a_in;
    a.cap = VT << LOG_T;                           // stage up to the consumers' capacity: records pack
    a.lay = make_engine_layout(a.cap, sizeof(K), staged_vsize(a), 1 << LOG_T, 4, 0);
    a.wait_ns = kWaitLimitNs;
    a.drop_fill = -1;
    constexpr int NG = kFusedConsumerGroups;
    auto kern = merge_engine_kernel<K, V, LOG_T, 4, 0, kSplitDiagonal, VT, true, NG>;
    if (!ensure_smem_limit(kern, a.lay.total)) return TM_ERR_UNSUPPORTED;
    const int block = (1 << LOG_T) * NG + 32;
    int per_sm = 0;
    if (const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, a.lay.total);
        e != cudaSuccess || per_sm < 1) {
        if (e != cudaSuccess) { record_cuda_error(e); cudaGetLastError(); }
        return TM_ERR_UNSUPPORTED;
    }
    const int64_t grid = (int64_t)per_sm * sm_count();
    // one grab per CTA where possible: its records pack into fuller tiles
    const int64_t g = (a.n_items + grid - 1) / grid;
    a.grab = (int)(g < 1 ? 1 : (g > 16 ? 16 : g));
    // Under stream capture the cooperative kernel goes in as an explicit graph
    // node (cooperative is a valid kernel-node attribute) after the stream's
    // current capture dependencies, which it then replaces.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (const cudaError_t e = cudaStreamIsCapturing(s, &cs); e != cudaSuccess) return cuda_failed(e);
    if (cs == cudaStreamCaptureStatusActive) {
        cudaGraph_t graph = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &graph, &deps, nullptr, &ndeps);
        if (e != cudaSuccess) return cuda_failed(e);
        void* args[1] = {&a};
        cudaKernelNodeParams kp = {};
        kp.func = reinterpret_cast<void*>(kern);
        kp.gridDim = dim3((unsigned)grid);
        kp.blockDim = dim3((unsigned)block);
        kp.sharedMemBytes = a.lay.total;
        kp.kernelParams = args;
        cudaGraphNode_t node = nullptr;
        if ((e = cudaGraphAddKernelNode(&node, graph, deps, ndeps, &kp)) != cudaSuccess) return cuda_failed(e);
        cudaKernelNodeAttrValue v = {};
        v.cooperative = 1;
        if ((e = cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributeCooperative, &v)) != cudaSuccess)
            return cuda_failed(e);
        e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
        return e == cudaSuccess ? TM_OK : cuda_failed(e);
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3((unsigned)block);
    lc.dynamicSmemBytes = a.lay.total;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&lc, kern, a);
    if (e == cudaErrorCooperativeLaunchTooLarge) {   // fewer SMs free than the occupancy says:
        cudaGetLastError();                           // the caller takes the separate launches
        return TM_ERR_UNSUPPORTED;
    }
    return e == cudaSuccess ? TM_OK : cuda_failed(e);
}

template <typename K, typename V>
tm_status launch_engine_fused_v(const EngineArgs& a, cudaStream_t s) {
    if (a.cap < 1) return TM_ERR_UNSUPPORTED;
    if (a.cap <= 9 * 128) return launch_fused_vt<K, V, 9>(a, s);
    if (a.cap <= 17 * 128) return launch_fused_vt<K, V, 17>(a, s);
    return TM_ERR_UNSUPPORTED;
}

template <typename K, typename V>
tm_status launch_engine_v(const EngineArgs& a, const tm_config* cfg, cudaStream_t s) {
    if (a.cap < 1 || a.cap > kMaxTileElems) return TM_ERR_UNSUPPORTED;
    const int split = (cfg && cfg->split) ? cfg->split : TM_SPLIT_DEFAULT;
    const int lt = log2_threads(cfg);
    if (a.Cv == nullptr) {                         // keys only: the diagonal split alone handles it
        if (split != TM_SPLIT_DIAGONAL) return TM_ERR_UNSUPPORTED;
        if (lt == 7 && a.cap <= 33 * 128) return launch_diagonal<K, V, 7>(a, cfg, s);
        if (lt == 8 && a.cap <= 33 * 256) return launch_diagonal<K, V, 8>(a, cfg, s);
        return TM_ERR_UNSUPPORTED;
    }
    if (split == TM_SPLIT_BLOCKS) {
        switch (lt) {
            case 7: return launch_blocks<K, V, 7>(a, cfg, s);
            case 8: return launch_blocks<K, V, 8>(a, cfg, s);
            case 9: return launch_blocks<K, V, 9>(a, cfg, s);
        }
    } else if (split == TM_SPLIT_DIAGONAL) {
        // tiles longer than 33 runs per thread fall back to the paper's rule
        if (lt == 7 && a.cap <= 33 * 128) return launch_diagonal<K, V, 7>(a, cfg, s);
        if (lt == 8 && a.cap <= 33 * 256) return launch_diagonal<K, V, 8>(a, cfg, s);
        switch (lt) {
            case 7: return launch_blocks<K, V, 7>(a, cfg, s);
            case 8: return launch_blocks<K, V, 8>(a, cfg, s);
            case 9: return launch_blocks<K, V, 9>(a, cfg, s);
        }
    }
    return TM_ERR_UNSUPPORTED;
}

// The 8-byte-payload launches; instantiated in their own translation units
// (tm_engine_<type>_v64.cu) so that they compile in parallel.
template <typename K>
tm_status launch_engine_v64(const EngineArgs& a, const tm_config* cfg, cudaStream_t s) {
    return launch_engine_v<K, uint64_t>(a, cfg, s);
}
template <typename K>
tm_status launch_engine_fused_v64(const EngineArgs& a, cudaStream_t s) {
    return launch_engine_fused_v<K, uint64_t>(a, s);
}

// Keys-only launches (Cv NULL) take the 4-byte instantiation: they stage no
// payloads, so the payload type does not matter.
template <typename K>
tm_status launch_engine(const EngineArgs& a, const tm_config* cfg, cudaStream_t s) {
    if (a.Cv != nullptr && a.vbytes == 8) return launch_engine_v64<K>(a, cfg, s);
    if (a.Cv != nullptr && a.vbytes != 4) return TM_ERR_UNSUPPORTED;
    return launch_engine_v<K, uint32_t>(a, cfg, s);
}

template <typename K>
tm_status launch_engine_fused(const EngineArgs& a, cudaStream_t s) {
    if (a.Cv != nullptr && a.vbytes == 8) return launch_engine_fused_v64<K>(a, s);
    if (a.Cv != nullptr && a.vbytes != 4) return TM_ERR_UNSUPPORTED;
    return launch_engine_fused_v<K, uint32_t>(a, s);
}

}  // namespace pmerge
