// Host-side launch of the four-run tile engine (two fused merge-sort
// rounds): pipeline depth and grid from the tile capacity, the key and
// payload sizes and the device's shared memory.  Instantiated per key type
// in tm_engine4_<type>.cu.
#pragma once

#include "tm_engine4.cuh"
#include "tm_host.h"

namespace pmerge {

template <typename K, typename V, int LOG_T, int S_IN, int VT>
tm_status launch_engine4_s(const Engine4Args& a_in, const tm_config* cfg, cudaStream_t s) {
    Engine4Args a = a_in;
    a.lay = make_engine4_layout(a.cap, sizeof(K), a.Cv ? (int)sizeof(V) : 0, S_IN);
    a.wait_ns = (cfg && cfg->wait_ms > 0) ? (uint64_t)cfg->wait_ms * 1000000ull : kWaitLimitNs;
    auto kern = merge4_engine_kernel<K, V, LOG_T, S_IN, VT>;
    if (!ensure_smem_limit(kern, a.lay.total)) return TM_ERR_UNSUPPORTED;
    const int block = (1 << LOG_T) + 32;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, a.lay.total) != cudaSuccess || per_sm < 1)
        return TM_ERR_UNSUPPORTED;
    int64_t grid = (int64_t)per_sm * sm_count();
    if (cfg && cfg->grid > 0) grid = cfg->grid;
    int64_t g = a.n_items / (grid * 8);
    a.grab = (int)(g < 1 ? 1 : (g > 16 ? 16 : g));
    const int64_t need = (a.n_items + a.grab - 1) / a.grab;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    if (cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s) != cudaSuccess) return TM_ERR_CUDA;
    kern<<<(unsigned)grid, block, a.lay.total, s>>>(a);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TM_OK : cuda_failed(e);
}

// 3 input stages when they fit the device's shared memory, else 2.
template <typename K, typename V, int LOG_T, int VT>
tm_status launch_engine4_vt(const Engine4Args& a, const tm_config* cfg, cudaStream_t s) {
    const int vs = a.Cv ? (int)sizeof(V) : 0;
    if (make_engine4_layout(a.cap, sizeof(K), vs, 3).total <= device_smem_limit())
        return launch_engine4_s<K, V, LOG_T, 3, VT>(a, cfg, s);
    return launch_engine4_s<K, V, LOG_T, 2, VT>(a, cfg, s);
}

// kEngine4LogT consumer threads (512: the two serial merge levels of a
// tile need many warps to hide their shared-memory latency); the smallest
// odd run length VT in {5, 9, 17, 33} with T VT >= cap.
constexpr int kEngine4LogT = 9;

template <typename K, typename V>
tm_status launch_engine4_v(const Engine4Args& a, const tm_config* cfg, cudaStream_t s) {
    constexpr int LT = kEngine4LogT, T = 1 << LT;
    if (a.cap < 1) return TM_ERR_UNSUPPORTED;
    if (a.cap <= 5 * T) return launch_engine4_vt<K, V, LT, 5>(a, cfg, s);
    if (a.cap <= 9 * T) return launch_engine4_vt<K, V, LT, 9>(a, cfg, s);
    if (a.cap <= 17 * T) return launch_engine4_vt<K, V, LT, 17>(a, cfg, s);
    if (a.cap <= 33 * T) return launch_engine4_vt<K, V, LT, 33>(a, cfg, s);
    return TM_ERR_UNSUPPORTED;
}

// vbytes: 4 or 8 (keys-only launches, Cv NULL, take the 4-byte instantiation).
template <typename K>
tm_status launch_engine4(const Engine4Args& a, int vbytes, const tm_config* cfg, cudaStream_t s) {
    if (a.Cv != nullptr && vbytes == 8) return launch_engine4_v<K, uint64_t>(a, cfg, s);
    return launch_engine4_v<K, uint32_t>(a, cfg, s);
}

}  // namespace pmerge
