// Host-side constants and helpers shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/tm.h"

namespace pmerge {

constexpr int kVersion = 1;
constexpr int kDefaultTile = 4096;        // elements of one staged subproblem
constexpr int kDefaultThreads = 256;      // threads per tile-merge CTA
constexpr int kMaxThreads = 512;          // launch bound of the tile kernels
constexpr int kMaxTileElems = 16384;      // cap on capA + capB
constexpr size_t kStatusBytes = 256;      // status word + padding at the head of a workspace
constexpr uint32_t kMaxSmemBytes = 232448;  // 227 KB opt-in dynamic shared memory per CTA

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline bool aligned(const void* p, size_t a) {
    return p != nullptr && (reinterpret_cast<uintptr_t>(p) % a) == 0;
}

// Opt-in dynamic shared memory per CTA of the current device, capped at
// kMaxSmemBytes.
inline uint32_t device_smem_limit() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    return (uint32_t)v < kMaxSmemBytes ? (uint32_t)v : kMaxSmemBytes;
}

// Raises a kernel's dynamic shared-memory limit to `bytes` (once per device
// and kernel, to the device's maximum); false if `bytes` does not fit.
template <typename Kernel>
inline bool ensure_smem_limit(Kernel kernel, uint32_t bytes) {
    static std::mutex mu;
    static uint64_t done_mask = 0;
    static uint32_t limit[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return false;
    std::lock_guard<std::mutex> lock(mu);
    if (!((done_mask >> dev) & 1ull)) {
        uint32_t lim = device_smem_limit();
        if (lim == 0) return false;
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim) != cudaSuccess)
            return false;
        limit[dev] = lim;
        done_mask |= 1ull << dev;
    }
    return bytes <= limit[dev];
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
size_t merge_workspace_bytes(int64_t p);

}  // namespace pmerge
