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
}  // extern "C"

// Steps 3-4 selection of all 2p subproblems (A side then B side) and each
// one's chain index, as the batched plan kernel computes them, in index
// type I: out[5k .. 5k+4] = a0, a1, b0, b1, chain.
template <typename I>
static void all_subproblems(I n, I m, I p, const int64_t* xbar, const int64_t* ybar, int64_t* out) {
    auto xb = [&](I i) { return (I)xbar[i]; };
    auto yb = [&](I j) { return (I)ybar[j]; };
    for (int side = 0; side < 2; ++side)
        for (I pe = 0; pe < p; ++pe) {
            I a0, a1, b0, b1;
            pmerge::subproblem_of<I>(side == 0, pe, n, m, p, xb, yb, a0, a1, b0, b1);
            const I chain = side == 0 ? pe + pmerge::first_block_at_or_after<I>(m, p, xb(pe))
                                      : pe + pmerge::first_block_at_or_after<I>(n, p, yb(pe));
            int64_t* o = out + 5 * ((int64_t)side * p + pe);
            o[0] = a0; o[1] = a1; o[2] = b0; o[3] = b1; o[4] = chain;
        }
}
extern "C" {
void h_all_subproblems32(int32_t n, int32_t m, int32_t p, const int64_t* xbar, const int64_t* ybar, int64_t* out) {
    all_subproblems<int32_t>(n, m, p, xbar, ybar, out);
}
void h_all_subproblems64(int64_t n, int64_t m, int64_t p, const int64_t* xbar, const int64_t* ybar, int64_t* out) {
    all_subproblems<int64_t>(n, m, p, xbar, ybar, out);
}
}
