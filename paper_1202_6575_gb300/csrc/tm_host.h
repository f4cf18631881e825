// Host-side constants and helpers shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <unordered_map>

#include <cuda_runtime.h>

#include "tm.h"

namespace pmerge {

constexpr int kVersion = 1;
constexpr int kDefaultTile = 2048;        // elements of one staged tile
constexpr int kDefaultThreads = 128;      // consumer threads per tile-merge CTA
constexpr int kMaxThreads = 512;          // launch bound of the tile kernels
constexpr int kMaxTileElems = 16384;      // cap on capA + capB
constexpr size_t kStatusBytes = 256;      // status word + padding at the head of a workspace
constexpr uint32_t kMaxSmemBytes = 232448;  // 227 KB opt-in dynamic shared memory per CTA

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline bool aligned(const void* p, size_t a) {
    return p != nullptr && (reinterpret_cast<uintptr_t>(p) % a) == 0;
}

// The CUDA error behind the calling thread's last TM_ERR_CUDA (see
// tm_last_cuda_error); cuda_failed records it and returns TM_ERR_CUDA.
void record_cuda_error(cudaError_t e);
inline tm_status cuda_failed(cudaError_t e) {
    record_cuda_error(e);
    return TM_ERR_CUDA;
}

// Payload arguments of a merge of n and m elements into C: all three
// arrays (each 4-byte aligned when its side is not empty), or, for a
// keys-only merge, none (the output payload pointer NULL, and so the input
// ones).
inline bool payloads_ok(int64_t n, const void* a, int64_t m, const void* b, const void* c, int vsize = 4) {
    if (c == nullptr) return a == nullptr && b == nullptr;
    return (n == 0 || aligned(a, vsize)) && (m == 0 || aligned(b, vsize)) && aligned(c, vsize);
}

// Bytes of one payload word selected by cfg (tm_config.payload_bytes: 0 or 4
// -> 4, 8 -> 8), -1 for anything else.
inline int payload_size(const tm_config* cfg) {
    const int b = cfg ? cfg->payload_bytes : 0;
    return b == 0 ? 4 : ((b == 4 || b == 8) ? b : -1);
}

// Opt-in dynamic shared memory per CTA of the current device, capped at
// kMaxSmemBytes.
inline uint32_t device_smem_limit() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    return (uint32_t)v < kMaxSmemBytes ? (uint32_t)v : kMaxSmemBytes;
}

// Raises a kernel's dynamic shared-memory limit to the device maximum less
// the kernel's static shared memory (once per kernel and device); false if
// `bytes` does not fit.
template <typename Kernel>
inline bool ensure_smem_limit(Kernel kernel, uint32_t bytes) {
    static std::mutex mu;
    static std::unordered_map<const void*, uint64_t> done;   // kernel -> device mask
    static std::unordered_map<const void*, uint32_t> limit;  // kernel -> its dynamic limit
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lock(mu);
    const void* key = reinterpret_cast<const void*>(kernel);
    uint64_t& mask = done[key];
    if (!((mask >> dev) & 1ull)) {
        cudaFuncAttributes fa{};
        cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
        const uint32_t dev_lim = device_smem_limit();
        const uint32_t lim = dev_lim > fa.sharedSizeBytes ? dev_lim - (uint32_t)fa.sharedSizeBytes : 0;
        if (e == cudaSuccess && lim > 0)
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
        if (e != cudaSuccess || lim == 0) {
            if (e != cudaSuccess) record_cuda_error(e);
            cudaGetLastError();                          // not sticky: later launches must not see it
            return false;
        }
        limit[key] = lim;                               // devices of one process share the part (sm_103a only)
        mask |= 1ull << dev;
    }
    return bytes <= limit[key];
}

// Streaming multiprocessors of the current device (cached per device).
inline int sm_count() {
    static std::mutex mu;
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 64 && cached[dev] > 0) return cached[dev];
    int n = 1;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (dev < 64) cached[dev] = n;
    return n;
}

int64_t choose_blocks(int64_t n, int64_t m, const tm_config* cfg);
int choose_threads(const tm_config* cfg);
size_t merge_workspace_bytes(int64_t p, const tm_config* cfg);
int log2_threads(const tm_config* cfg);
tm_status merge_tiles_dispatch(tm_key_type kt, const void* a_keys, const uint32_t* a_vals, int64_t n,
                               const void* b_keys, const uint32_t* b_vals, int64_t m,
                               const void* tiles, int64_t n_tiles, int cap,
                               void* c_keys, uint32_t* c_vals, void* control,
                               const tm_config* cfg, cudaStream_t s);

}  // namespace pmerge
