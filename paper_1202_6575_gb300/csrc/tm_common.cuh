// Shared device helpers of the stable parallel merge (sm_103a).
//
// Notation follows Traeff, "Simplified, stable parallel merging", Section 2:
// A[0..n), B[0..m) non-decreasing, p blocks per array, block starts x_i / y_j
// (the first len mod p blocks one element longer), cross ranks
// xbar_i = rank_low(A[x_i], B) and ybar_j = rank_high(B[y_j], A).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "tm.h"

namespace pmerge {

// ---------------------------------------------------------------------------
// Key types
// ---------------------------------------------------------------------------
// Native C++ '<' gives exactly the orders of the ABI: unsigned for uint32_t
// and uint64_t, signed for int32_t, IEEE for float (-0.0 == +0.0).

template <typename K> struct KeyOf;
template <> struct KeyOf<uint32_t> { static constexpr tm_key_type id = TM_KEY_U32; };
template <> struct KeyOf<int32_t>  { static constexpr tm_key_type id = TM_KEY_I32; };
template <> struct KeyOf<uint64_t> { static constexpr tm_key_type id = TM_KEY_U64; };
template <> struct KeyOf<float>    { static constexpr tm_key_type id = TM_KEY_F32; };

inline size_t key_size(tm_key_type kt) { return (kt == TM_KEY_U64) ? 8 : 4; }

// ---------------------------------------------------------------------------
// Block decomposition (Section 2)
// ---------------------------------------------------------------------------

// a / b for 0 <= a, 0 < b: a 32-bit division when both operands fit (the
// usual case: blocks and tiles of one merge), else the full-width one.
template <typename I>
__host__ __device__ __forceinline__ I div_nonneg(I a, I b) {
    if (sizeof(I) > 4 && ((uint64_t)a | (uint64_t)b) <= 0xffffffffull) return (I)((uint32_t)a / (uint32_t)b);
    return a / b;
}

// x_i for 0 <= i <= p: i*ceil(len/p) for i < r = len mod p, else
// i*floor(len/p) + r (so x_p = len).
template <typename I>
__host__ __device__ __forceinline__ I block_start(I len, I p, I i) {
    I q = div_nonneg(len, p), r = len - q * p;
    return (i < r) ? i * (q + 1) : i * q + r;
}

// Block holding index k (0 <= k <= len); k = len is "block p".  The O(1)
// rule of Section 2, with the empty-block case (floor(len/p) = 0) covered by
// k >= r*ceil(len/p) = len.
template <typename I>
__host__ __device__ __forceinline__ I block_of(I len, I p, I k) {
    if (k >= len) return p;
    I q = div_nonneg(len, p), r = len - q * p;
    I head = r * (q + 1);
    return (k < head) ? div_nonneg(k, q + 1) : div_nonneg(k - head, q) + r;
}

// Smallest block index j whose start y_j is >= k (0 <= k <= len): the block
// of k, or the next one when k lies strictly inside its block.  For k = len
// that is the first empty block (index len when len < p), else block p.
template <typename I>
__host__ __device__ __forceinline__ I first_block_at_or_after(I len, I p, I k) {
    if (k >= len) return len < p ? len : p;
    I j = block_of(len, p, k);
    return (block_start(len, p, j) == k) ? j : j + 1;
}

// Division by an invariant divisor (Lemire, Kaser and Kurz, "Faster
// remainder by direct computation", 2019): for x, d < 2^32 and d > 1,
// floor(x / d) is the high 64 bits of the 128-bit product c * x with
// c = ceil(2^64 / d).  d = 1 returns x.
struct FastDiv32 {
    uint64_t c;
    uint32_t d;
    __host__ __device__ FastDiv32() : c(0), d(1) {}
    __host__ __device__ explicit FastDiv32(uint32_t dd) : c(dd > 1 ? ~0ull / dd + 1 : 0), d(dd) {}
    __host__ __device__ __forceinline__ uint32_t div(uint32_t x) const {
        if (d <= 1) return x;
#ifdef __CUDA_ARCH__
        return (uint32_t)__umul64hi(c, (uint64_t)x);
#else
        return (uint32_t)(((unsigned __int128)c * x) >> 64);
#endif
    }
};

// The block decomposition of Section 2 for len + p < 2^32, with its
// parameters computed once: q = floor(len / p), r = len mod p (the first r
// blocks one longer), head = r (q + 1) = the end of the longer blocks.
// Same values as block_start / block_of / first_block_at_or_after.
struct Blocks32 {
    uint32_t len, p, q, r, head;
    FastDiv32 dq1, dq;                              // division by q + 1 and by q
    __host__ __device__ Blocks32() : len(0), p(1), q(0), r(0), head(0) {}
    __host__ __device__ Blocks32(uint32_t len_, uint32_t p_)
        : len(len_), p(p_), q(len_ / p_), r(len_ % p_), head((len_ % p_) * (len_ / p_ + 1)),
          dq1(len_ / p_ + 1), dq(len_ / p_) {}
    // x_i for 0 <= i <= p
    __host__ __device__ __forceinline__ int64_t start(int64_t i) const {
        const uint32_t u = (uint32_t)i;
        return (int64_t)(u < r ? u * (q + 1) : u * q + r);
    }
    // block holding index k (0 <= k <= len); k = len -> p
    __host__ __device__ __forceinline__ int64_t of(int64_t k) const {
        const uint32_t u = (uint32_t)k;
        if (u >= len) return p;
        return (int64_t)(u < head ? dq1.div(u) : dq.div(u - head) + r);
    }
    // smallest block index whose start is >= k (0 <= k <= len)
    __host__ __device__ __forceinline__ int64_t first_at_or_after(int64_t k) const {
        if ((uint32_t)k >= len) return len < p ? len : p;
        const int64_t j = of(k);
        return start(j) == k ? j : j + 1;
    }
};

// The same decomposition through the general functions above (any length).
template <typename I>
struct BlocksOf {
    I len, p;
    __host__ __device__ __forceinline__ I start(I i) const { return block_start<I>(len, p, i); }
    __host__ __device__ __forceinline__ I first_at_or_after(I k) const { return first_block_at_or_after<I>(len, p, k); }
};

// ---------------------------------------------------------------------------
// Rank primitives (Section 2)
// ---------------------------------------------------------------------------
// rank_low(x, X)  = #{k : X[k] <  x}  (the i with X[i-1] <  x <= X[i])
// rank_high(x, X) = #{k : X[k] <= x}  (the j with X[j-1] <= x <  X[j])

template <typename K, typename I>
__device__ __forceinline__ I rank_low_global(const K* __restrict__ X, I len, K x) {
    I lo = 0;
    while (len > 0) {
        I half = len >> 1;
        if (__ldg(X + lo + half) < x) { lo += half + 1; len -= half + 1; }
        else                           { len = half; }
    }
    return lo;
}

template <typename K, typename I>
__device__ __forceinline__ I rank_high_global(const K* __restrict__ X, I len, K x) {
    I lo = 0;
    while (len > 0) {
        I half = len >> 1;
        if (!(x < __ldg(X + lo + half))) { lo += half + 1; len -= half + 1; }
        else                             { len = half; }
    }
    return lo;
}

template <typename K>
__device__ __forceinline__ int rank_low_smem(const K* X, int len, K x) {
    int lo = 0;
    while (len > 0) {
        int half = len >> 1;
        if (X[lo + half] < x) { lo += half + 1; len -= half + 1; }
        else                  { len = half; }
    }
    return lo;
}

template <typename K>
__device__ __forceinline__ int rank_high_smem(const K* X, int len, K x) {
    int lo = 0;
    while (len > 0) {
        int half = len >> 1;
        if (!(x < X[lo + half])) { lo += half + 1; len -= half + 1; }
        else                     { len = half; }
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Subproblem of one processing element, by the split-point form of Steps 3-4
// ---------------------------------------------------------------------------
// The points P_A(i) = (x_i, xbar_i), P_B(j) = (ybar_j, y_j) and (n, m) lie on
// the merge path and, by Observation 1, form one chain ordered by a + b (the
// output offset).  The subproblem of A-PE i runs from P_A(i) to the next
// point of the chain: P_B(j') with j' the first B block starting at or after
// xbar_i, if y_j' < xbar_{i+1}, else P_A(i+1).  This is exactly cases (a)-(e)
// of Step 3:  (a) xbar_i = xbar_{i+1} -> no B point between;  (e) xbar_i = y_j
// -> next is P_B(j);  (b)/(d) -> P_A(i+1);  (c) -> P_B(j+1).  Step 4 is the
// mirror.  Returns the A range [a0, a1), B range [b0, b1); the output starts
// at a0 + b0.

// bA, bB: the block decompositions of A and B (start(i), first_at_or_after(k)).
template <typename I, typename BA, typename BB, typename LoadXbar, typename LoadYbar>
__host__ __device__ __forceinline__ void subproblem_in(bool a_side, I pe, I p, const BA& bA, const BB& bB,
                                                       LoadXbar xbar, LoadYbar ybar, I& a0, I& a1, I& b0, I& b1) {
    if (a_side) {
        I xi = bA.start(pe), xi1 = bA.start(pe + 1);
        I xb = xbar(pe), xb1 = xbar(pe + 1);
        a0 = xi; b0 = xb;
        I jn = bB.first_at_or_after(xb);
        I yjn = bB.start(jn);
        if (jn < p && yjn < xb1) { a1 = ybar(jn); b1 = yjn; }
        else                     { a1 = xi1;      b1 = xb1; }
    } else {
        I yj = bB.start(pe), yj1 = bB.start(pe + 1);
        I yb = ybar(pe), yb1 = ybar(pe + 1);
        b0 = yj; a0 = yb;
        I in = bA.first_at_or_after(yb);
        I xin = bA.start(in);
        if (in < p && xin < yb1) { b1 = xbar(in); a1 = xin; }
        else                     { b1 = yj1;      a1 = yb1; }
    }
}

template <typename I, typename LoadXbar, typename LoadYbar>
__host__ __device__ __forceinline__ void subproblem_of(bool a_side, I pe, I n, I m, I p,
                                                       LoadXbar xbar, LoadYbar ybar,
                                                       I& a0, I& a1, I& b0, I& b1) {
    subproblem_in<I>(a_side, pe, p, BlocksOf<I>{n, p}, BlocksOf<I>{m, p}, xbar, ybar, a0, a1, b0, b1);
}

// ---------------------------------------------------------------------------
// Device status word
// ---------------------------------------------------------------------------

__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
    if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy (TMA engine) wrappers, inline PTX for sm_90+.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\t"
                 "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Waits for phase `parity` of the barrier; gives up after `limit_ns`
// nanoseconds of global time and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// Bulk global -> shared copy; completion is counted on `bar` in bytes.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gmem_src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(smem_dst)), "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// Bulk shared -> global copy in the current bulk group.
__device__ __forceinline__ void bulk_s2g(void* gmem_dst, const void* smem_src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                 :: "l"(gmem_dst), "r"(smem_u32(smem_src)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until at most N committed bulk groups still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" :: "n"(N) : "memory");
}

template <int N>
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group %0;" :: "n"(N) : "memory");
}

// Wait time for one tile's bulk loads before a kernel reports TM_ERR_TIMEOUT
// (a tile normally lands in microseconds).
constexpr uint64_t kWaitLimitNs = 2000000000ull;

}  // namespace pmerge
