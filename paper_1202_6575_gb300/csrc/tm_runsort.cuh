// Stable in-CTA sort of the merge sort's initial runs (Section 3: the p
// consecutive blocks are first sorted each on its own, with any stable
// sequential sort, and then merged).
//
// One CTA sorts one run of up to kSortRun elements by least-significant-
// digit radix sort on the keys' order-preserving unsigned images, 8 bits per
// pass.  LSD radix sort is stable: every pass keeps the order of equal
// digits, so equal keys keep their input order, as the stable merge rounds
// that follow require.  A pass over a digit window in which every key of the
// run agrees is the identity and is skipped, so a run costs one pass per
// byte in which its keys differ (three for keys below 2^24, eight at most
// for 64-bit keys); its cost per element does not grow with the run length,
// which is why the runs are 4096 long (two merge rounds fewer than runs of
// 1024).
//
// A pass: the elements sit at run positions 0..len-1; thread (warp w, lane l)
// holds items q = 0..VT-1 at positions w*32*VT + q*32 + l, so a warp's items
// in (q, lane) order are its positions in increasing order.  Each warp ranks
// its items among equal digits (the peers of one digit, from one ballot per
// digit bit; earlier lanes first) and keeps a running count per digit; one
// exclusive scan of the counts in (digit, warp) order then gives every
// digit's and warp's first output position, and each item lands at that
// position plus its rank.  Keys move through shared memory and registers;
// payloads only through shared memory (two buffers, each item's payload
// copied from its old position to its new one), which keeps them out of the
// registers during the ranking.  The counts are [warp][digit], so that the
// per-digit updates of one warp fall on distinct banks.
#pragma once
#include <cstdint>

namespace pmerge {

constexpr int kSortRun = 4096;
constexpr int kSortThreads = 256;                         // two CTAs per SM at 128 registers a thread
constexpr int kSortVT = kSortRun / kSortThreads;          // 16 items per thread
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kRadixBits = 8;
constexpr int kRadixDigits = 1 << kRadixBits;
constexpr int kScanPerThread = kRadixDigits * kSortWarps / kSortThreads;   // 8 counts per thread
static_assert(kSortRun == kSortThreads * kSortVT, "a run is VT items of every thread");
static_assert(kRadixDigits * kSortWarps == kSortThreads * kScanPerThread, "the scan splits evenly");

// Unsigned image of a key whose unsigned order is the key order of the merge
// ('<' of the key type): identity for unsigned keys, the sign bit flipped for
// int32, and for float the usual sign-magnitude flip after mapping -0.0 to
// +0.0 (they are equal keys, so they must get equal images).  NaN keys are
// not supported anywhere in the library.
template <typename K> struct RadixImage;
template <> struct RadixImage<uint32_t> {
    using U = uint32_t;
    __device__ __forceinline__ static U of(uint32_t k) { return k; }
};
template <> struct RadixImage<int32_t> {
    using U = uint32_t;
    __device__ __forceinline__ static U of(int32_t k) { return static_cast<uint32_t>(k) ^ 0x80000000u; }
};
template <> struct RadixImage<uint64_t> {
    using U = uint64_t;
    __device__ __forceinline__ static U of(uint64_t k) { return k; }
};
template <> struct RadixImage<float> {
    using U = uint32_t;
    __device__ __forceinline__ static U of(float k) {
        uint32_t u = __float_as_uint(k);
        if (u == 0x80000000u) u = 0u;
        return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    }
};

template <typename K, typename V>
constexpr uint32_t run_sort_smem_bytes() {
    return (uint32_t)(kSortRun * (sizeof(K) + 2 * sizeof(V)) + sizeof(int) * kRadixDigits * kSortWarps);
}

// The lanes of the warp whose digit equals this lane's, among the lanes with
// ok set (lanes without it get the set of such lanes, unused): one ballot
// per digit bit, and one for ok unless every lane has it (all_ok, the same
// for the whole warp).
__device__ __forceinline__ unsigned digit_peers(unsigned d, bool ok, bool all_ok) {
    unsigned m = 0xffffffffu;
    if (!all_ok) {
        m = __ballot_sync(0xffffffffu, ok);
        m = ok ? m : ~m;
    }
#pragma unroll
    for (int b = 0; b < kRadixBits; ++b) {
        const bool bit = (d >> b) & 1u;
        const unsigned v = __ballot_sync(0xffffffffu, bit);
        m &= ~(v ^ (0u - (unsigned)bit));             // v where the bit is set, ~v where clear
    }
    return m;
}

// Exclusive prefix sum over the CTA's threads (in thread order); `tot`
// holds kSortWarps ints of scratch.  Every thread must call it.
__device__ __forceinline__ int cta_exclusive_scan(int x, int* tot) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int t0 = lane < kSortWarps ? tot[lane] : 0;
        int ti = t0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < kSortWarps) tot[lane] = ti - t0;
    }
    __syncthreads();
    const int r = incl - x + tot[w];
    __syncthreads();                                   // tot is reused by the next call
    return r;
}

// One run X[base, base + len) (len <= kSortRun; FULL: len == kSortRun, so
// that no item needs a bounds check).
template <typename K, typename V, bool FULL>
__device__ __forceinline__ void run_sort_body(const K* __restrict__ in_k, const V* __restrict__ in_v,
                                              K* __restrict__ out_k, V* __restrict__ out_v, int64_t base,
                                              int len, uint8_t* smem) {
    using R = RadixImage<K>;
    using U = typename R::U;
    K* sk = reinterpret_cast<K*>(smem);
    V* sv = reinterpret_cast<V*>(smem + (size_t)kSortRun * sizeof(K));          // payloads, two buffers
    int* hist = reinterpret_cast<int*>(smem + (size_t)kSortRun * (sizeof(K) + 2 * sizeof(V)));  // [warp][digit]
    __shared__ U red[kSortWarps], red2[kSortWarps];
    __shared__ int tot[kSortWarps];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const bool vals = in_v != nullptr;
    const int p0 = w * 32 * kSortVT + lane;            // item q sits at p0 + 32 q
    const uint32_t lt_mask = (1u << lane) - 1u;
    auto has = [&](int q) { return FULL || p0 + 32 * q < len; };

    K k[kSortVT];
#pragma unroll
    for (int q = 0; q < kSortVT; ++q) {
        const int i = p0 + 32 * q;
        k[q] = K();
        if (has(q)) {
            k[q] = in_k[base + i];
            if (vals) sv[i] = in_v[base + i];
        }
    }
    int cur = 0;                                       // payload buffer holding the current order
    // the bits in which the run's keys differ: set in some key, clear in another
    U any = 0, all = ~(U)0;
#pragma unroll
    for (int q = 0; q < kSortVT; ++q)
        if (has(q)) {
            any |= R::of(k[q]);
            all &= R::of(k[q]);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        any |= __shfl_xor_sync(0xffffffffu, any, o);
        all &= __shfl_xor_sync(0xffffffffu, all, o);
    }
    if (lane == 0) { red[w] = any; red2[w] = all; }
    __syncthreads();
    any = 0;
    all = ~(U)0;
#pragma unroll
    for (int j = 0; j < kSortWarps; ++j) { any |= red[j]; all &= red2[j]; }
    const U diff = any ^ all;

    bool in_smem = false;                              // the current key order is in sk, not only in k
    int* hw = hist + w * kRadixDigits;
    for (int sh = 0; sh < (int)(8 * sizeof(U)); sh += kRadixBits) {
        if (((diff >> sh) & (U)(kRadixDigits - 1)) == 0) continue;   // same for the whole CTA
        if (in_smem) {
#pragma unroll
            for (int q = 0; q < kSortVT; ++q) {
                const int i = p0 + 32 * q;
                if (has(q)) k[q] = sk[i];
            }
        }
        for (int j = t; j < kRadixDigits * kSortWarps; j += kSortThreads) hist[j] = 0;
        __syncthreads();                               // counts zeroed; every read of sk done
        int dl[kSortVT];                               // digit << 16 | rank among the warp's earlier items of it
#pragma unroll
        for (int q = 0; q < kSortVT; ++q) {
            const bool ok = has(q);
            const int d = (int)((R::of(k[q]) >> sh) & (U)(kRadixDigits - 1));
            const unsigned peers = digit_peers((unsigned)d, ok, FULL);
            const int leader = __ffs(peers) - 1;
            int b = 0;
            if (ok && lane == leader) b = hw[d];
            b = __shfl_sync(0xffffffffu, b, leader);
            if (ok && lane == leader) hw[d] = b + __popc(peers);
            dl[q] = (d << 16) | (b + __popc(peers & lt_mask));
            __syncwarp();
        }
        __syncthreads();
        // exclusive scan of the counts in (digit, warp) order: thread t takes
        // scan positions [t S, (t+1) S), position s = digit * warps + warp
        int c[kScanPerThread];
        int sum = 0;
#pragma unroll
        for (int j = 0; j < kScanPerThread; ++j) {
            const int s = t * kScanPerThread + j;
            c[j] = hist[(s % kSortWarps) * kRadixDigits + s / kSortWarps];
            sum += c[j];
        }
        int run = cta_exclusive_scan(sum, tot);
#pragma unroll
        for (int j = 0; j < kScanPerThread; ++j) {
            const int s = t * kScanPerThread + j;
            hist[(s % kSortWarps) * kRadixDigits + s / kSortWarps] = run;
            run += c[j];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kSortVT; ++q) {
            if (has(q)) {
                const int dst = hw[dl[q] >> 16] + (dl[q] & 0xffff);
                sk[dst] = k[q];
                if (vals) sv[(cur ^ 1) * kSortRun + dst] = sv[cur * kSortRun + p0 + 32 * q];
            }
        }
        __syncthreads();
        in_smem = true;
        cur ^= 1;
    }
    if (in_smem) {
        for (int i = t; i < len; i += kSortThreads) {
            out_k[base + i] = sk[i];
            if (vals) out_v[base + i] = sv[cur * kSortRun + i];
        }
    } else {                                           // no pass: the run was already in order
#pragma unroll
        for (int q = 0; q < kSortVT; ++q) {
            const int i = p0 + 32 * q;
            if (has(q)) {
                out_k[base + i] = k[q];
                if (vals) out_v[base + i] = sv[i];
            }
        }
    }
}

// rdesc (optional): run b is X[rdesc[2b], rdesc[2b] + rdesc[2b+1]) (at most
// kSortRun elements); without it run b is X[b kSortRun, ...) clipped to n.
// in_v == nullptr (and out_v): keys only.  The run may be sorted in place
// (in == out).
template <typename K, typename V>
__global__ void __launch_bounds__(kSortThreads, 2)
run_sort_kernel(const K* __restrict__ in_k, const V* __restrict__ in_v, K* __restrict__ out_k,
                V* __restrict__ out_v, int64_t n, const int64_t* __restrict__ rdesc = nullptr) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int64_t base = rdesc ? __ldg(rdesc + 2 * blockIdx.x) : (int64_t)blockIdx.x * kSortRun;
    const int64_t rl = rdesc ? __ldg(rdesc + 2 * blockIdx.x + 1) : n - base;
    const int len = (int)(rl < kSortRun ? (rl > 0 ? rl : 0) : kSortRun);
    if (len == kSortRun) run_sort_body<K, V, true>(in_k, in_v, out_k, out_v, base, len, smem);
    else if (len > 0)    run_sort_body<K, V, false>(in_k, in_v, out_k, out_v, base, len, smem);
}

}  // namespace pmerge
