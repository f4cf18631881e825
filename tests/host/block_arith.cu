// Test harness: the library's block arithmetic (csrc/tm_common.cuh, the
// __host__ __device__ functions the kernels use for Section 2's block
// decomposition) compiled for the host, so that the CPU tests can compare it
// with the oracle at sizes no GPU test can allocate.  Built by
// tests/test_host_arith.py into a temporary directory; not part of libtm.
#include "tm_common.cuh"

extern "C" {
int64_t h_div_nonneg64(int64_t a, int64_t b) { return pmerge::div_nonneg<int64_t>(a, b); }
int32_t h_div_nonneg32(int32_t a, int32_t b) { return pmerge::div_nonneg<int32_t>(a, b); }
int64_t h_block_start64(int64_t len, int64_t p, int64_t i) { return pmerge::block_start<int64_t>(len, p, i); }
int32_t h_block_start32(int32_t len, int32_t p, int32_t i) { return pmerge::block_start<int32_t>(len, p, i); }
int64_t h_block_of64(int64_t len, int64_t p, int64_t k) { return pmerge::block_of<int64_t>(len, p, k); }
int64_t h_first_block64(int64_t len, int64_t p, int64_t k) {
    return pmerge::first_block_at_or_after<int64_t>(len, p, k);
}
uint32_t h_fastdiv32(uint32_t x, uint32_t d) { return pmerge::FastDiv32(d).div(x); }
int64_t h_blocks32_start(uint32_t len, uint32_t p, int64_t i) { return pmerge::Blocks32(len, p).start(i); }
int64_t h_blocks32_of(uint32_t len, uint32_t p, int64_t k) { return pmerge::Blocks32(len, p).of(k); }
int64_t h_blocks32_first(uint32_t len, uint32_t p, int64_t k) { return pmerge::Blocks32(len, p).first_at_or_after(k); }
}
