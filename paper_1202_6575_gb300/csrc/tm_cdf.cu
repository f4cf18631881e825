// Learned cross-rank proposal (not in the paper) for repeated merges into a
// large sorted base array, and its training kernels.
//
// Model (float32, in one caller-owned device buffer, layout in include/tm.h):
//   knot keys   K[0..S]: K[s] = X[R[s]] for s < S, K[S] = X[N-1], taken once
//               from the base X (N keys);
//   knot ranks  R[0..S]: positions of the knot keys in the current base
//               (R[s] = floor(s N / S) when built); kept in two buffers so a
//               merge can write the ranks for the merged base while reading
//               the current ones;
//   MLP         z = W1 [f0, f1] + b1 (H units), h = relu(z), y = w2 . h + b2,
//               on f0 = 2t - 1, f1 = (2s + 1)/S - 1, where s is the segment
//               of the key (number of K[1..S-1] <= key) and t its position
//               in the segment, clamped to [0, 1];
//   prediction  pred = R[s] + t (R[s+1] - R[s]) + y * max(R[s+1] - R[s], 1);
//   error bound eps_frac = max |y - tau| over the labelled keys, in units of
//               the segment's size (tau = (label - pla) / scale).
// Training minimises mean 0.5 (y - tau)^2 by full-batch Adam (beta 0.9,
// 0.999, eps 1e-8); labels are exact rank_high values that the plain search
// kernel computes.
//
// Use: the learned Steps 1-2 kernel proposes every cross rank from the model
// and searches only a window around the proposal, then verifies the answer
// against the definition of rank_low / rank_high (Section 2) with at most
// two extra probes; a failed check runs the plain full binary search.  The
// merged output is therefore exactly the plain method's, whatever the model.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>

#include "tm_engine.cuh"
#include "tm_host.h"

namespace pmerge {

// TM_OK, or TM_ERR_CUDA with the pending launch error recorded for
// tm_last_cuda_error.
static tm_status launch_status() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TM_OK : cuda_failed(e);
}

struct CdfHeader {
    int32_t S, H;
    float eps_frac;
    int32_t cur;                       // current knot-rank buffer (0 or 1)
    int64_t N;                         // base length the current ranks refer to
    unsigned long long fallbacks;      // learned searches that fell back to the full search
    unsigned long long learned;        // learned searches issued
    int64_t adam_step;
    float loss;
    uint32_t arrived;                  // CTAs of a learned search that finished reading the ranks (0 between calls)
};
// The byte layout include/tm.h documents for the model header (the binding
// reads it at these offsets).
static_assert(offsetof(CdfHeader, S) == 0 && offsetof(CdfHeader, H) == 4 && offsetof(CdfHeader, eps_frac) == 8 &&
              offsetof(CdfHeader, cur) == 12 && offsetof(CdfHeader, N) == 16 &&
              offsetof(CdfHeader, fallbacks) == 24 && offsetof(CdfHeader, learned) == 32 &&
              offsetof(CdfHeader, adam_step) == 40 && offsetof(CdfHeader, loss) == 48 &&
              offsetof(CdfHeader, arrived) == 52 && sizeof(CdfHeader) <= 256,
              "model header layout differs from the one documented in tm.h");

struct CdfLayout {
    size_t K, R0, R1, params, m, v, grad, eps_seg, bytes;
};

__host__ __device__ inline size_t a256(size_t x) { return (x + 255) / 256 * 256; }

__host__ __device__ inline CdfLayout cdf_layout(int S, int H) {
    CdfLayout L;
    const size_t P = 4 * (size_t)H + 1;
    size_t o = 256;
    L.K = o; o += a256((S + 1) * sizeof(float));
    L.R0 = o; o += a256((S + 1) * sizeof(int64_t));
    L.R1 = o; o += a256((S + 1) * sizeof(int64_t));
    L.params = o; o += a256(P * sizeof(float));
    L.m = o; o += a256(P * sizeof(float));
    L.v = o; o += a256(P * sizeof(float));
    L.grad = o; o += a256(P * sizeof(float));
    L.eps_seg = o; o += a256((size_t)S * sizeof(float));
    L.bytes = o;
    return L;
}

// View of a model on the device.  The current rank buffer is chosen on the
// device from the header (cur), so no call needs to read the header back.
struct CdfView {
    const CdfHeader* hdr;
    const float* K;
    int64_t* R0;
    int64_t* R1;
    const float* params;               // W1 (H x 2), b1 (H), w2 (H), b2
    float* eps_seg;                    // per-segment error bound (segment units), 0 = no labels seen
    int S, H;
    __device__ __forceinline__ const int64_t* ranks() const { return hdr->cur ? R1 : R0; }
    __device__ __forceinline__ int64_t* next_ranks() const { return hdr->cur ? R0 : R1; }
};

__device__ __forceinline__ int cdf_segment(const float* K, int S, float q) {
    // number of interior knots K[1..S-1] that are <= q
    int lo = 0, len = S - 1;
    const float* X = K + 1;
    while (len > 0) {
        int half = len >> 1;
        if (!(q < __ldg(X + lo + half))) { lo += half + 1; len -= half + 1; } else { len = half; }
    }
    return lo;
}

// Features, PLA part and the segment's rank scale of key q.
struct CdfPoint {
    int s;
    float t, f0, f1;
    double pla, scale;
};

__device__ __forceinline__ CdfPoint cdf_point(const float* K, const int64_t* R, int S, float q) {
    CdfPoint c;
    c.s = cdf_segment(K, S, q);
    const float k0 = __ldg(K + c.s), k1 = __ldg(K + c.s + 1);
    const float w = k1 - k0;
    float t = (w > 0.f) ? (q - k0) / w : 0.f;
    t = fminf(fmaxf(t, 0.f), 1.f);
    c.t = t;
    c.f0 = 2.f * t - 1.f;
    c.f1 = (2.f * c.s + 1.f) / (float)S - 1.f;
    const int64_t r0 = R[c.s], r1 = R[c.s + 1];
    const double seg = (double)(r1 - r0);
    c.pla = (double)r0 + (double)t * seg;
    c.scale = seg > 1.0 ? seg : 1.0;
    return c;
}

// MLP output y for features (f0, f1); params in shared memory.
__device__ __forceinline__ float cdf_mlp(const float* p, int H, float f0, float f1) {
    const float* W1 = p;
    const float* b1 = p + 2 * H;
    const float* w2 = p + 3 * H;
    float y = p[4 * H];
    for (int k = 0; k < H; ++k) {
        const float z = fmaf(W1[2 * k], f0, fmaf(W1[2 * k + 1], f1, b1[k]));
        y = fmaf(w2[k], fmaxf(z, 0.f), y);
    }
    return y;
}

// ---------------------------------------------------------------------------
// Build and training kernels
// ---------------------------------------------------------------------------

__global__ void cdf_knots_kernel(const float* __restrict__ X, int64_t N, int S, float* __restrict__ K,
                                 int64_t* __restrict__ R) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s > S) return;
    const int64_t r = (s < S) ? ((int64_t)s * N) / S : N;
    R[s] = r;
    K[s] = (s < S) ? X[r] : X[N - 1];
}

__global__ void cdf_init_kernel(CdfHeader* h, int S, int H, int64_t N, float* params, const float* init,
                                float* m, float* v, float* grad) {
    const int P = 4 * H + 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        params[i] = init[i];
        m[i] = 0.f; v[i] = 0.f; grad[i] = 0.f;
    }
    if (threadIdx.x == 0) {
        h->S = S; h->H = H; h->eps_frac = 0.f; h->cur = 0; h->N = N;
        h->fallbacks = 0; h->learned = 0; h->adam_step = 0; h->loss = 0.f; h->arrived = 0;
    }
}

// Forward + backward of the mean half-squared residual over `count` labelled
// keys; gradients accumulate into grad[0..P) and the loss into h->loss
// (both zeroed by the caller).  One query per thread (grid-stride); each
// hidden unit's four gradient terms are warp-reduced, then added to shared
// accumulators, then once per CTA to global memory.
__global__ void __launch_bounds__(256)
cdf_grad_kernel(CdfView mv, const float* __restrict__ q, const int64_t* __restrict__ labels, int64_t count,
                float* __restrict__ grad, CdfHeader* hdr) {
    extern __shared__ float sm[];
    const int H = mv.H, P = 4 * H + 1;
    float* p = sm;                 // params
    float* acc = sm + P;           // gradient accumulators
    __shared__ float sloss;
    for (int i = threadIdx.x; i < P; i += blockDim.x) { p[i] = mv.params[i]; acc[i] = 0.f; }
    if (threadIdx.x == 0) sloss = 0.f;
    __syncthreads();
    const float invB = 1.f / (float)count;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t start = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t iters = (count + stride - 1) / stride;   // same trip count for the whole warp
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t i = start + it * stride;
        const bool valid = i < count;
        float f0 = 0.f, f1 = 0.f, dy = 0.f, l = 0.f;
        if (valid) {
            const CdfPoint c = cdf_point(mv.K, mv.ranks(), mv.S, q[i]);
            f0 = c.f0; f1 = c.f1;
            const float y = cdf_mlp(p, H, f0, f1);
            const float tau = (float)(((double)labels[i] - c.pla) / c.scale);
            const float r = y - tau;
            dy = r * invB;
            l = 0.5f * r * r * invB;
        }
        for (int k = 0; k < H; ++k) {
            const float z = fmaf(p[2 * k], f0, fmaf(p[2 * k + 1], f1, p[2 * H + k]));
            const float hk = fmaxf(z, 0.f);
            const float dz = (z > 0.f) ? dy * p[3 * H + k] : 0.f;
            float g0 = dz * f0, g1 = dz * f1, gb = dz, gw = dy * hk;
            for (int o = 16; o > 0; o >>= 1) {
                g0 += __shfl_xor_sync(0xffffffffu, g0, o);
                g1 += __shfl_xor_sync(0xffffffffu, g1, o);
                gb += __shfl_xor_sync(0xffffffffu, gb, o);
                gw += __shfl_xor_sync(0xffffffffu, gw, o);
            }
            if (lane == 0) {
                atomicAdd(&acc[2 * k], g0);
                atomicAdd(&acc[2 * k + 1], g1);
                atomicAdd(&acc[2 * H + k], gb);
                atomicAdd(&acc[3 * H + k], gw);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            dy += __shfl_xor_sync(0xffffffffu, dy, o);
            l += __shfl_xor_sync(0xffffffffu, l, o);
        }
        if (lane == 0) { atomicAdd(&acc[4 * H], dy); atomicAdd(&sloss, l); }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P; i += blockDim.x) atomicAdd(&grad[i], acc[i]);
    if (threadIdx.x == 0) atomicAdd(&hdr->loss, sloss);
}

// One Adam update of all P parameters (single CTA); zeroes the gradient.
__global__ void cdf_adam_kernel(CdfHeader* h, float* params, float* m, float* v, float* grad, int P, float lr) {
    __shared__ int64_t step;
    if (threadIdx.x == 0) step = h->adam_step + 1;
    __syncthreads();
    const double c1 = 1.0 - pow(0.9, (double)step), c2 = 1.0 - pow(0.999, (double)step);
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const float g = grad[i];
        const float mi = 0.9f * m[i] + 0.1f * g;
        const float vi = 0.999f * v[i] + 0.001f * g * g;
        m[i] = mi; v[i] = vi;
        const float mh = (float)(mi / c1), vh = (float)(vi / c2);
        params[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
        grad[i] = 0.f;
    }
    __syncthreads();
    if (threadIdx.x == 0) h->adam_step = step;
}

__global__ void __launch_bounds__(256)
cdf_predict_kernel(CdfView mv, const float* __restrict__ q, int64_t count, float* __restrict__ pred,
                   float* __restrict__ resid, const int64_t* __restrict__ labels, CdfHeader* hdr) {
    extern __shared__ float sm[];
    const int P = 4 * mv.H + 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) sm[i] = mv.params[i];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const CdfPoint c = cdf_point(mv.K, mv.ranks(), mv.S, q[i]);
    const float y = cdf_mlp(sm, mv.H, c.f0, c.f1);
    if (pred) pred[i] = (float)(c.pla + (double)y * c.scale);
    if (labels) {                                   // |y - tau| for the error bounds
        const float tau = (float)(((double)labels[i] - c.pla) / c.scale);
        const float e = fabsf(y - tau);
        if (resid) resid[i] = e;
        // e >= 0, so the int order of its bits is the float order
        atomicMax(reinterpret_cast<int*>(&hdr->eps_frac), __float_as_int(e));
        atomicMax(reinterpret_cast<int*>(&mv.eps_seg[c.s]), __float_as_int(e));
    }
}

// ---------------------------------------------------------------------------
// Learned Steps 1-2 for A = the base (the model's array, n keys) and B = an
// incoming batch (m keys); flags bit 0: also write the knot ranks of the
// merged base into the other rank buffer (R_next[s] = R[s] + rank_low(K[s],
// B): the knot element moves by the B keys placed before it).
// ---------------------------------------------------------------------------

// Verified window search: the unique r with X[r-1] < x <= X[r] (rank_low,
// HIGH = false) or X[r-1] <= x < X[r] (rank_high) searched in [lo, hi]; if the
// window does not bracket it (checked against the definition, at most two
// probes), a full binary search.  Returns true when the window sufficed.
//
// Inside the window the probes are placed from the data.  A bracket [a, b]
// holds the answer whenever the window does: a probe at q reads X[q-1] and
// either raises a to q (X[q-1] lies before x, so r >= q) or lowers b to q-1.
// Any choice of q keeps that invariant, so the placement below affects only
// the number of memory sectors touched, never the result:
//   1. one probe at the model's estimate r0 + off;
//   2. from its key, the estimate moves by (x - key) * rho (rho = base
//      elements per key unit of the segment) and two probes bracket it at
//      2.5 standard deviations of the count of elements in that key range
//      (about sqrt of the move) plus 3;
//   3. when both bracket ends have known keys, linear interpolation between
//      them and two probes 4 elements either side;
// then bisection of what is left (usually one 32-byte sector).
template <bool HIGH>
__device__ __forceinline__ bool guided_rank(const float* __restrict__ X, int64_t len, float x, int64_t lo,
                                            int64_t hi, int64_t r0, float off, float rho, int64_t& r) {
    auto before = [&](float v) { return HIGH ? !(x < v) : (v < x); };   // v belongs before x
    int64_t a = lo, b = hi;
    float ka = 0.f, kb = 0.f;                          // keys of X[a-1] and X[b] once probed
    bool has_a = false, has_b = false;
    auto clampq = [&](int64_t q) { return q <= a ? a + 1 : (q > b ? b : q); };
    auto apply = [&](int64_t q, float v) {
        if (before(v)) { if (q > a) { a = q; ka = v; has_a = true; } }
        else if (q - 1 < b) { b = q - 1; kb = v; has_b = true; }
    };
    if (b > a) {                                       // 1. the model's estimate
        const int64_t q1 = clampq(r0 + (int64_t)rintf(fminf(fmaxf(off, -2e9f), 2e9f)));
        const float v1 = __ldg(X + q1 - 1);
        apply(q1, v1);
        if (b > a) {                                   // 2. local density from the segment
            const float dr = (x - v1) * rho;
            const float g = 2.5f * sqrtf(fabsf(dr)) + 3.f;
            const float lo_off = fmaxf(dr - g, -2e9f), hi_off = fminf(dr + g, 2e9f);
            const int64_t q2 = clampq(q1 + (int64_t)floorf(lo_off));
            const int64_t q3 = clampq(q1 + (int64_t)ceilf(hi_off));
            const float v2 = __ldg(X + q2 - 1), v3 = __ldg(X + q3 - 1);
            apply(q2, v2);
            apply(q3, v3);
        }
        if (b - a > 8 && has_a && has_b && kb > ka) {  // 3. interpolation between the bracket's keys
            const float f = fminf(fmaxf((x - ka) / (kb - ka), 0.f), 1.f);
            const int64_t c = a + (int64_t)(f * (float)(b - a + 1));
            const int64_t q4 = clampq(c - 4), q5 = clampq(c + 4);
            const float v4 = __ldg(X + q4 - 1), v5 = __ldg(X + q5 - 1);
            apply(q4, v4);
            apply(q5, v5);
        }
    }
    int64_t l = b - a;
    while (l > 0) {
        const int64_t h = l >> 1;
        if (before(__ldg(X + a + h))) { a += h + 1; l -= h + 1; } else { l = h; }
    }
    const bool ok_lo = (a > lo) || a == 0 || before(__ldg(X + a - 1));
    const bool ok_hi = (a < hi) || a == len || !before(__ldg(X + a));
    if (ok_lo && ok_hi) { r = a; return true; }
    r = HIGH ? rank_high_global<float, int64_t>(X, len, x) : rank_low_global<float, int64_t>(X, len, x);
    return false;
}

// ---------------------------------------------------------------------------
// Search-side evaluation of the model, in float32 and integer arithmetic
// only (no float64 on the search path): the proposal is r0 + off with
// r0 = R[s] exact and off = t * seg + y * max(seg, 1) a float offset.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int segment_of_key(const float* __restrict__ K, int S, float q) {
    int lo = 0, len = S - 1;                           // knots K[1..S-1] <= q
    const float* X = K + 1;
    while (len > 0) {
        const int half = len >> 1;
        if (!(q < __ldg(X + lo + half))) { lo += half + 1; len -= half + 1; } else { len = half; }
    }
    return lo;
}

// MLP output for features (f0, f1) from parameters staged per hidden unit
// as {W1[k][0], W1[k][1], b1[k], w2[k]} (one 16-byte shared load per unit),
// four independent partial sums.
__device__ __forceinline__ float mlp_units(const float4* __restrict__ u, float b2, int H, float f0, float f1) {
    float y0 = b2, y1 = 0.f, y2 = 0.f, y3 = 0.f;
    int k = 0;
    for (; k + 4 <= H; k += 4) {
        const float4 a = u[k], b = u[k + 1], c = u[k + 2], d = u[k + 3];
        y0 = fmaf(a.w, fmaxf(fmaf(a.x, f0, fmaf(a.y, f1, a.z)), 0.f), y0);
        y1 = fmaf(b.w, fmaxf(fmaf(b.x, f0, fmaf(b.y, f1, b.z)), 0.f), y1);
        y2 = fmaf(c.w, fmaxf(fmaf(c.x, f0, fmaf(c.y, f1, c.z)), 0.f), y2);
        y3 = fmaf(d.w, fmaxf(fmaf(d.x, f0, fmaf(d.y, f1, d.z)), 0.f), y3);
    }
    for (; k < H; ++k) {
        const float4 a = u[k];
        y0 = fmaf(a.w, fmaxf(fmaf(a.x, f0, fmaf(a.y, f1, a.z)), 0.f), y0);
    }
    return (y0 + y1) + (y2 + y3);
}

// Proposal for key q: r0 (exact rank of the segment's left knot), the float
// offset from it, and the window half-width in base ranks (three times the
// segment's calibrated error, the global one when the segment saw no
// labels, plus a margin: a single fallback in a launch of ~10^5 searches
// puts a full search on the launch's critical path, and doubling the window
// costs one probe), and rho, the segment's base elements per key unit (the
// local density that guides the probes inside the window).
struct Proposal { int64_t r0; float off, w, rho; };

__device__ __forceinline__ Proposal propose(const float* __restrict__ K, const float4* __restrict__ units, float b2,
                                            const CdfView& mv, const int64_t* R,
                                            float eps_global, float q) {
    const int S = mv.S;
    const int s = segment_of_key(K, S, q);
    const float k0 = __ldg(K + s), k1 = __ldg(K + s + 1);
    const float wk = k1 - k0;
    float t = (wk > 0.f) ? (q - k0) / wk : 0.f;
    t = fminf(fmaxf(t, 0.f), 1.f);
    const int64_t r0 = R[s];
    const float seg = (float)(R[s + 1] - r0);
    const float scale = fmaxf(seg, 1.f);
    const float y = mlp_units(units, b2, mv.H, 2.f * t - 1.f, (2.f * s + 1.f) / (float)S - 1.f);
    float e = mv.eps_seg[s];
    if (!(e > 0.f)) e = eps_global;
    Proposal pr;
    pr.r0 = r0;
    pr.off = t * seg + y * scale;
    pr.w = 3.f * e * scale + 32.f;
    pr.rho = (wk > 0.f) ? seg / wk : 0.f;
    return pr;
}

// Window around the exact base rank r0 + off (float offset only: no loss of
// precision for ranks beyond 2^24).
__device__ __forceinline__ void base_window(const Proposal& pr, int64_t n, int64_t& lo, int64_t& hi) {
    const int64_t a = pr.r0 + (int64_t)floorf(fminf(fmaxf(pr.off - pr.w, -4e9f), 4e9f));
    const int64_t b = pr.r0 + (int64_t)ceilf(fminf(fmaxf(pr.off + pr.w, -4e9f), 4e9f));
    lo = a < 0 ? 0 : (a > n ? n : a);
    hi = b < 0 ? 0 : (b > n ? n : b);
    if (lo > hi) lo = hi;
}

// Steps 1-2 with the model on the searches into the base.  The A-block
// starts search the batch B and the knot updates search B too: B is small
// and the upper levels of those bisections are shared by all threads and
// stay in L2, so they use the plain bisection.  The B-block starts search
// the large base A, where every bisection ends in ~8 distinct DRAM sectors:
// there the model's window and the data-guided probes inside it replace the
// descent (~5 sectors).  Those searches are the longest, so they take the
// first thread indices (the first CTAs to be scheduled).  The knots are read
// through L1 (16 KB, shared by every CTA on an SM); the MLP parameters are
// staged in shared memory, one float4 per hidden unit.
__global__ void __launch_bounds__(256, 8)
learned_cross_rank_kernel(CdfView mv, CdfHeader* hdr, const float* __restrict__ A, int64_t n,
                          const float* __restrict__ B, int64_t m, int64_t p, int64_t* __restrict__ xbar,
                          int64_t* __restrict__ ybar, int advance) {
    extern __shared__ float4 units[];                  // MLP parameters, one float4 per hidden unit
    const int H = mv.H;
    for (int k = threadIdx.x; k < H; k += blockDim.x)
        units[k] = make_float4(mv.params[2 * k], mv.params[2 * k + 1], mv.params[2 * H + k], mv.params[3 * H + k]);
    const float b2 = mv.params[4 * H];
    __syncthreads();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float eps = hdr->eps_frac;
    const int64_t* R = mv.ranks();
    int fell = 0, used = 0;
    if (t < p) {                                       // B-side: rank_high(B[y_j], A) in the base
        const int64_t j = t;
        const int64_t yj = block_start<int64_t>(m, p, j);
        int64_t r = n;
        if (yj < m) {
            const float key = __ldg(B + yj);
            const Proposal pr = propose(mv.K, units, b2, mv, R, eps, key);
            int64_t lo, hi;
            base_window(pr, n, lo, hi);
            fell = !guided_rank<true>(A, n, key, lo, hi, pr.r0, pr.off, pr.rho, r);
            used = 1;
        }
        ybar[j] = r;
    } else if (t < 2 * p) {                            // A-side: rank_low(A[x_i], B)
        const int64_t i = t - p;
        const int64_t xi = block_start<int64_t>(n, p, i);
        xbar[i] = (xi < n) ? rank_low_global<float, int64_t>(B, m, __ldg(A + xi)) : m;
    } else if (t == 2 * p) {
        xbar[p] = m;
        ybar[p] = n;
    } else if (advance && t <= 2 * p + 1 + mv.S) {     // knot ranks of the merged base
        const int s = (int)(t - 2 * p - 1);
        mv.next_ranks()[s] = R[s] + (s < mv.S ? rank_low_global<float, int64_t>(B, m, __ldg(mv.K + s)) : m);
    }
    // warp-aggregated counters
    const unsigned f = __ballot_sync(0xffffffffu, fell), u = __ballot_sync(0xffffffffu, used);
    if ((threadIdx.x & 31) == 0) {
        if (f) atomicAdd(&hdr->fallbacks, (unsigned long long)__popc(f));
        if (u) atomicAdd(&hdr->learned, (unsigned long long)__popc(u));
    }
    if (advance) {                                     // the last CTA to finish makes the new ranks current
        __syncthreads();                               // this CTA's reads of the current ranks are done
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(&hdr->arrived, 1u) == gridDim.x - 1) {
                __threadfence();
                hdr->cur ^= 1;
                hdr->N = n + m;
                hdr->arrived = 0;
            }
        }
    }
}

}  // namespace pmerge

using namespace pmerge;

namespace {

bool cdf_dims_ok(int S, int H) { return S >= 2 && S <= (1 << 20) && H >= 1 && H <= 1024; }

CdfView cdf_view(void* model, int S, int H) {
    const CdfLayout L = cdf_layout(S, H);
    uint8_t* b = static_cast<uint8_t*>(model);
    CdfView v;
    v.hdr = reinterpret_cast<const CdfHeader*>(b);
    v.K = reinterpret_cast<const float*>(b + L.K);
    v.R0 = reinterpret_cast<int64_t*>(b + L.R0);
    v.R1 = reinterpret_cast<int64_t*>(b + L.R1);
    v.params = reinterpret_cast<const float*>(b + L.params);
    v.eps_seg = reinterpret_cast<float*>(b + L.eps_seg);
    v.S = S; v.H = H;
    return v;
}

bool model_ok(const void* model, int S, int H) { return cdf_dims_ok(S, H) && aligned(model, 256); }

}  // namespace

extern "C" {

size_t tm_cdf_model_bytes(int segments, int hidden) {
    if (!cdf_dims_ok(segments, hidden)) return 0;
    return cdf_layout(segments, hidden).bytes;
}

tm_status tm_cdf_init(void* model, int segments, int hidden, const float* base_keys, int64_t n,
                      const float* init_params, tm_stream_t stream) {
    if (!model_ok(model, segments, hidden) || n < 1 || !aligned(base_keys, 4) || !aligned(init_params, 4))
        return TM_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const CdfLayout L = cdf_layout(segments, hidden);
    uint8_t* b = static_cast<uint8_t*>(model);
    cdf_knots_kernel<<<(segments + 256) / 256, 256, 0, s>>>(base_keys, n, segments, reinterpret_cast<float*>(b + L.K),
                                                          reinterpret_cast<int64_t*>(b + L.R0));
    if (const cudaError_t e_ = cudaMemsetAsync(b + L.eps_seg, 0, (size_t)segments * sizeof(float), s); e_ != cudaSuccess) return cuda_failed(e_);
    cdf_init_kernel<<<1, 256, 0, s>>>(reinterpret_cast<CdfHeader*>(b), segments, hidden, n,
                                      reinterpret_cast<float*>(b + L.params), init_params,
                                      reinterpret_cast<float*>(b + L.m), reinterpret_cast<float*>(b + L.v),
                                      reinterpret_cast<float*>(b + L.grad));
    return launch_status();
}

tm_status tm_cdf_grad(void* model, int segments, int hidden, const float* q, const int64_t* labels, int64_t count,
                      float* grad_out, float* loss_out, tm_stream_t stream) {
    if (!model_ok(model, segments, hidden) || count < 1 || !aligned(q, 4) || !aligned(labels, 8) ||
        !aligned(grad_out, 4) || !aligned(loss_out, 4))
        return TM_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const CdfLayout L = cdf_layout(segments, hidden);
    const int P = 4 * hidden + 1;
    CdfHeader* hdr = static_cast<CdfHeader*>(model);
    CdfView v = cdf_view(model, segments, hidden);
    float* g = reinterpret_cast<float*>(static_cast<uint8_t*>(model) + L.grad);
    if (const cudaError_t e_ = cudaMemsetAsync(g, 0, P * sizeof(float), s); e_ != cudaSuccess) return cuda_failed(e_);
    if (const cudaError_t e_ = cudaMemsetAsync(&hdr->loss, 0, sizeof(float), s); e_ != cudaSuccess) return cuda_failed(e_);
    const int64_t blocks = std::min<int64_t>((count + 255) / 256, 4096);
    cdf_grad_kernel<<<(unsigned)blocks, 256, 2 * P * sizeof(float), s>>>(v, q, labels, count, g, hdr);
    if (const tm_status st = launch_status(); st != TM_OK) return st;
    cudaError_t e = cudaMemcpyAsync(grad_out, g, P * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss_out, &hdr->loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g, 0, P * sizeof(float), s);
    return e == cudaSuccess ? TM_OK : cuda_failed(e);
}

tm_status tm_cdf_train(void* model, int segments, int hidden, const float* q, const int64_t* labels, int64_t count,
                       int steps, float lr, tm_stream_t stream) {
    if (!model_ok(model, segments, hidden) || count < 1 || steps < 0 || !aligned(q, 4) || !aligned(labels, 8) ||
        !(lr > 0.f))
        return TM_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const CdfLayout L = cdf_layout(segments, hidden);
    const int P = 4 * hidden + 1;
    uint8_t* b = static_cast<uint8_t*>(model);
    CdfHeader* hdr = reinterpret_cast<CdfHeader*>(b);
    CdfView v = cdf_view(model, segments, hidden);
    float* g = reinterpret_cast<float*>(b + L.grad);
    const int64_t blocks = std::min<int64_t>((count + 255) / 256, 4096);
    if (const cudaError_t e_ = cudaMemsetAsync(g, 0, P * sizeof(float), s); e_ != cudaSuccess) return cuda_failed(e_);
    for (int it = 0; it < steps; ++it) {
        if (const cudaError_t e_ = cudaMemsetAsync(&hdr->loss, 0, sizeof(float), s); e_ != cudaSuccess) return cuda_failed(e_);
        cdf_grad_kernel<<<(unsigned)blocks, 256, 2 * P * sizeof(float), s>>>(v, q, labels, count, g, hdr);
        cdf_adam_kernel<<<1, 288, 0, s>>>(hdr, reinterpret_cast<float*>(b + L.params), reinterpret_cast<float*>(b + L.m),
                                          reinterpret_cast<float*>(b + L.v), g, P, lr);
    }
    return launch_status();
}

tm_status tm_cdf_predict(const void* model, int segments, int hidden, const float* q, int64_t count, float* pred,
                         tm_stream_t stream) {
    if (!model_ok(model, segments, hidden) || count < 0 || !aligned(q, 4) || !aligned(pred, 4))
        return TM_ERR_INVALID;
    if (count == 0) return TM_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int P = 4 * hidden + 1;
    CdfView v = cdf_view(const_cast<void*>(model), segments, hidden);
    cdf_predict_kernel<<<(unsigned)((count + 255) / 256), 256, P * sizeof(float), s>>>(
        v, q, count, pred, nullptr, nullptr, const_cast<CdfHeader*>(v.hdr));
    return launch_status();
}

tm_status tm_cdf_calibrate(void* model, int segments, int hidden, const float* q, const int64_t* labels,
                           int64_t count, tm_stream_t stream) {
    if (!model_ok(model, segments, hidden) || count < 1 || !aligned(q, 4) || !aligned(labels, 8))
        return TM_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int P = 4 * hidden + 1;
    CdfHeader* hdr = static_cast<CdfHeader*>(model);
    CdfView v = cdf_view(model, segments, hidden);
    if (const cudaError_t e_ = cudaMemsetAsync(&hdr->eps_frac, 0, sizeof(float), s); e_ != cudaSuccess) return cuda_failed(e_);
    if (const cudaError_t e_ = cudaMemsetAsync(v.eps_seg, 0, (size_t)segments * sizeof(float), s); e_ != cudaSuccess) return cuda_failed(e_);
    cdf_predict_kernel<<<(unsigned)((count + 255) / 256), 256, P * sizeof(float), s>>>(
        v, q, count, nullptr, nullptr, labels, hdr);
    return launch_status();
}

tm_status tm_cross_ranks_learned(void* model, int segments, int hidden, const float* a_keys, int64_t n,
                                 const float* b_keys, int64_t m, int64_t p, int64_t* xbar, int64_t* ybar,
                                 int flags, tm_stream_t stream) {
    if (!model_ok(model, segments, hidden) || n < 1 || m < 0 || p < 1 || !aligned(a_keys, 4) ||
        (m > 0 && !aligned(b_keys, 4)) || !aligned(xbar, 8) || !aligned(ybar, 8))
        return TM_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CdfView v = cdf_view(model, segments, hidden);
    const int64_t threads = 2 * p + 2 + segments;
    learned_cross_rank_kernel<<<(unsigned)((threads + 255) / 256), 256, (size_t)hidden * sizeof(float4), s>>>(
        v, static_cast<CdfHeader*>(model), a_keys, n, b_keys, m, p, xbar, ybar, flags & TM_LEARNED_ADVANCE);
    if (const tm_status st_ = launch_status(); st_ != TM_OK) return st_;

    return TM_OK;
}

tm_status tm_merge_learned(void* model, int segments, int hidden,
                           const float* a_keys, const uint32_t* a_vals, int64_t n,
                           const float* b_keys, const uint32_t* b_vals, int64_t m,
                           float* c_keys, uint32_t* c_vals, void* workspace, size_t workspace_bytes,
                           const tm_config* cfg, int flags, tm_stream_t stream) {
    // every argument rule of the calls below, checked before anything is issued
    if (!model_ok(model, segments, hidden) || n < 1 || m < 0) return TM_ERR_INVALID;
    if (payload_size(cfg) != 4) return TM_ERR_UNSUPPORTED;
    if (!aligned(a_keys, 4) || (m > 0 && !aligned(b_keys, 4)) || !aligned(c_keys, 4) ||
        !payloads_ok(n, a_vals, m, b_vals, c_vals))
        return TM_ERR_INVALID;
    const int64_t p = choose_blocks(n, m, cfg);
    if (!workspace || !aligned(workspace, 256) || workspace_bytes < merge_workspace_bytes(p, cfg))
        return TM_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the workspace layout of tm_merge: control | xbar | ybar | tiles
    uint8_t* w = static_cast<uint8_t*>(workspace);
    int64_t* xbar = reinterpret_cast<int64_t*>(w + kStatusBytes);
    int64_t* ybar = reinterpret_cast<int64_t*>(w + kStatusBytes + align_up((size_t)(p + 1) * 8, 256));
    void* tiles = w + kStatusBytes + 2 * align_up((size_t)(p + 1) * 8, 256);
    if (const cudaError_t e_ = cudaMemsetAsync(w, 0, sizeof(int32_t), s); e_ != cudaSuccess) return cuda_failed(e_);
    tm_status st = tm_cross_ranks_learned(model, segments, hidden, a_keys, n, b_keys, m, p, xbar, ybar, flags,
                                          stream);
    if (st != TM_OK) return st;
    st = tm_plan_subproblems(n, m, p, xbar, ybar, tiles, cfg, stream);
    if (st != TM_OK) return st;
    return tm_merge_tiles(TM_KEY_F32, a_keys, a_vals, n, b_keys, b_vals, m, tiles, tm_plan_tile_count(n, m, p),
                          tm_merge_tile_cap(n, m, p), c_keys, c_vals, workspace, cfg, stream);
}

}  // extern "C"
