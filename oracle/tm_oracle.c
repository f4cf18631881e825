/*
 * Reference oracle for the stable parallel merge of Traeff, "Simplified,
 * stable parallel merging" (arXiv:1202.6575).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * CPU statement of what the GPU library computes.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark load it.  It shares no
 * code, header, table or helper with the CUDA library, and the library never
 * calls it.
 *
 * Everything here is single-threaded, written for readability, and follows
 * the paper's notation (paper_parallel.c, a CPU baseline, runs the same
 * steps on several threads):
 *   A[0..n), B[0..m)   non-decreasing inputs (Section 2), sentinels
 *                      A[-1] = -inf, A[n] = +inf are implied, never stored;
 *   rank_low(x, X)     the unique i with X[i-1] < x <= X[i]  (Section 2);
 *   rank_high(x, X)    the unique j with X[j-1] <= x < X[j]  (Section 2);
 *   x_i, y_j           block starts, first n mod p blocks one longer
 *                      (Section 2, block decomposition), x_p = n, y_p = m;
 *   xbar_i, ybar_j     cross ranks (Steps 1 and 2);
 *   Steps 3 and 4      the five cases (a)-(e) and their B-side mirror.
 *
 * Payloads are opaque 32-bit words that travel with their keys.
 *
 * Readings of the paper taken here (the paper is silent or garbled there):
 *   - case (d) of Step 3 reads "A[x_i .. x_{i+1}-1]" (the text prints
 *     x_{j+1}; the correctness argument of Section 2 and Figure 1's y_0 and
 *     y_3 subproblems fix the index);
 *   - Step 4 is Step 3 with A<->B, x<->y, xbar<->ybar exchanged;
 *   - the index len (one past the end) belongs to "block p", whose start is
 *     x_p = len; this makes "different blocks" well defined when a cross rank
 *     equals len;
 *   - when p > len the first len blocks hold one element and the rest are
 *     empty with start len; the key at an empty block's start is the +inf
 *     sentinel, so its cross rank is the full length of the other array;
 *   - ties: every A element precedes every equal B element, each side keeps
 *     its input order (Section 2, stability); inputs are never swapped.
 *
 * Key types: u32 and u64 compare unsigned, i32 signed, f32 by IEEE '<'
 * (inputs carry no NaN).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------- */
/* Block decomposition (Section 2).  Type independent.                     */
/* ---------------------------------------------------------------------- */

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

/* x_i for 0 <= i <= p: i*ceil(len/p) for i < r = len mod p, otherwise
 * i*floor(len/p) + r.  For i = p this gives len, i.e. x_p = n. */
int64_t orc_block_start(int64_t len, int64_t p, int64_t i)
{
    int64_t r = len % p;
    if (i < r) return i * ceil_div(len, p);
    return i * (len / p) + r;
}

/* The block index k (0 <= k <= len) belongs to, by the paper's O(1) rule:
 * k < r*ceil(len/p)  ->  floor(k / ceil(len/p)),
 * otherwise          ->  floor((k - r*ceil(len/p)) / floor(len/p)) + r.
 * k = len is "block p" (one past the last block). */
int64_t orc_block_of(int64_t len, int64_t p, int64_t k)
{
    if (k >= len) return p;
    int64_t r = len % p;
    int64_t c = ceil_div(len, p);
    if (k < r * c) return k / c;
    return (k - r * c) / (len / p) + r;
}

/* ---------------------------------------------------------------------- */
/* Steps 3 and 4: the five cases.  Type independent: they read only the     */
/* block starts and the cross ranks.                                         */
/*                                                                           */
/* Output: table[6*k + 0..5] = {lo, hi, other_lo, other_hi, c_lo, case}     */
/* for k = 0..2p-1, where rows 0..p-1 are the A-side processing elements     */
/* (lo..hi is an A range, other_lo..other_hi a B range) and rows p..2p-1     */
/* the B-side ones (lo..hi a B range, other a A range).  c_lo is the first   */
/* output index; case is 'a'..'e'.  Ranges are half open.                    */
/* ---------------------------------------------------------------------- */

static void one_side_case(int64_t len_own, int64_t len_oth, int64_t p, int64_t i,
                          const int64_t* bar_own, const int64_t* bar_oth, int64_t* row)
{
    /* Processing element i of the "own" array (A in Step 3, B in Step 4).
     * bar_own[i] is the cross rank of own[x_i] in the other array;
     * bar_oth[j] is the cross rank of oth[y_j] in the own array. */
    int64_t xi  = orc_block_start(len_own, p, i);
    int64_t xi1 = orc_block_start(len_own, p, i + 1);
    int64_t xb  = bar_own[i];
    int64_t xb1 = bar_own[i + 1];
    int64_t c0  = xi + xb;

    /* (a) both cross ranks equal: the whole own block goes out alone. */
    if (xb == xb1) {
        row[0] = xi; row[1] = xi1; row[2] = xb; row[3] = xb; row[4] = c0; row[5] = 'a';
        return;
    }
    int64_t j  = orc_block_of(len_oth, p, xb);
    int64_t yj = orc_block_start(len_oth, p, j);
    /* (e) xbar_i is exactly the start of block j of the other array: the own
     *     elements before ybar_j go out alone. */
    if (xb == yj) {
        row[0] = xi; row[1] = bar_oth[j]; row[2] = xb; row[3] = xb; row[4] = c0; row[5] = 'e';
        return;
    }
    int64_t j1  = orc_block_of(len_oth, p, xb1);
    int64_t yj1 = orc_block_start(len_oth, p, j + 1);
    /* (b) both cross ranks inside the same block j. */
    if (j1 == j) {
        row[0] = xi; row[1] = xi1; row[2] = xb; row[3] = xb1; row[4] = c0; row[5] = 'b';
        return;
    }
    /* Different blocks, xbar_i strictly inside block j. */
    if (xb1 != yj1) {
        /* (c) stop at the next block start y_{j+1}; the own range ends at
         *     ybar_{j+1}, which lies inside own block i. */
        row[0] = xi; row[1] = bar_oth[j + 1]; row[2] = xb; row[3] = yj1; row[4] = c0; row[5] = 'c';
        return;
    }
    /* (d) xbar_{i+1} = y_{j+1}: the whole own block meets B[xbar_i .. y_{j+1}). */
    row[0] = xi; row[1] = xi1; row[2] = xb; row[3] = yj1; row[4] = c0; row[5] = 'd';
}

/* Subproblem k of the 2p: A-side PE k (Step 3) for k < p, else B-side PE
 * k - p (Step 4, roles exchanged; row[4] = y_j + ybar_j, own start + own
 * cross rank). */
void orc_subproblem(int64_t n, int64_t m, int64_t p, int64_t k,
                    const int64_t* xbar, const int64_t* ybar, int64_t* row)
{
    if (k < p) one_side_case(n, m, p, k, xbar, ybar, row);
    else       one_side_case(m, n, p, k - p, ybar, xbar, row);
}

void orc_subproblems(int64_t n, int64_t m, int64_t p,
                     const int64_t* xbar, const int64_t* ybar, int64_t* table)
{
    for (int64_t k = 0; k < 2 * p; ++k)
        orc_subproblem(n, m, p, k, xbar, ybar, table + 6 * k);
}

/* ---------------------------------------------------------------------- */
/* Typed parts, instantiated once per key type.                              */
/* ---------------------------------------------------------------------- */

#define DEFINE_ORACLE(S, T)                                                           \
                                                                                      \
/* rank_low(x, X): the unique i, 0 <= i <= len, with X[i-1] < x <= X[i]          */  \
/* (sentinels X[-1] = -inf, X[len] = +inf).  Binary search for the first        */  \
/* index whose element is not below x.                                          */  \
int64_t orc_rank_low_##S(T x, const T* X, int64_t len)                                \
{                                                                                     \
    int64_t lo = 0, hi = len;          /* answer in [lo, hi] */                       \
    while (lo < hi) {                                                                 \
        int64_t mid = lo + (hi - lo) / 2;                                             \
        if (X[mid] < x) lo = mid + 1; else hi = mid;                                  \
    }                                                                                 \
    return lo;                                                                        \
}                                                                                     \
                                                                                      \
/* rank_high(x, X): the unique j with X[j-1] <= x < X[j].                       */  \
int64_t orc_rank_high_##S(T x, const T* X, int64_t len)                               \
{                                                                                     \
    int64_t lo = 0, hi = len;                                                         \
    while (lo < hi) {                                                                 \
        int64_t mid = lo + (hi - lo) / 2;                                             \
        if (!(x < X[mid])) lo = mid + 1; else hi = mid;                               \
    }                                                                                 \
    return lo;                                                                        \
}                                                                                     \
                                                                                      \
/* Textbook stable two-way merge: B[j] is taken only when B[j] < A[i],          */  \
/* so on equal keys A comes first.                                              */  \
void orc_merge_two_pointer_##S(const T* A, const uint32_t* Av, int64_t n,             \
                               const T* B, const uint32_t* Bv, int64_t m,             \
                               T* C, uint32_t* Cv)                                    \
{                                                                                     \
    int64_t i = 0, j = 0, k = 0;                                                      \
    while (i < n && j < m) {                                                          \
        if (B[j] < A[i]) { C[k] = B[j]; Cv[k] = Bv[j]; ++j; }                         \
        else             { C[k] = A[i]; Cv[k] = Av[i]; ++i; }                         \
        ++k;                                                                          \
    }                                                                                 \
    while (i < n) { C[k] = A[i]; Cv[k] = Av[i]; ++i; ++k; }                           \
    while (j < m) { C[k] = B[j]; Cv[k] = Bv[j]; ++j; ++k; }                           \
}                                                                                     \
                                                                                      \
/* The position formulas of Section 2: A[i] lands at i + rank_low(A[i], B),     */  \
/* B[j] at j + rank_high(B[j], A).                                              */  \
void orc_merge_rank_scatter_##S(const T* A, const uint32_t* Av, int64_t n,            \
                                const T* B, const uint32_t* Bv, int64_t m,            \
                                T* C, uint32_t* Cv)                                   \
{                                                                                     \
    for (int64_t i = 0; i < n; ++i) {                                                 \
        int64_t pos = i + orc_rank_low_##S(A[i], B, m);                               \
        C[pos] = A[i]; Cv[pos] = Av[i];                                               \
    }                                                                                 \
    for (int64_t j = 0; j < m; ++j) {                                                 \
        int64_t pos = j + orc_rank_high_##S(B[j], A, n);                              \
        C[pos] = B[j]; Cv[pos] = Bv[j];                                               \
    }                                                                                 \
}                                                                                     \
                                                                                      \
/* Steps 1 and 2: xbar_i = rank_low(A[x_i], B) for i < p, xbar_p = m;           */  \
/* ybar_j = rank_high(B[y_j], A) for j < p, ybar_p = n.  An empty block's start */  \
/* is the +inf sentinel, whose ranks are m and n.                               */  \
void orc_cross_ranks_##S(const T* A, int64_t n, const T* B, int64_t m, int64_t p,     \
                         int64_t* xbar, int64_t* ybar)                                \
{                                                                                     \
    for (int64_t i = 0; i < p; ++i) {                                                 \
        int64_t xi = orc_block_start(n, p, i);                                        \
        xbar[i] = (xi < n) ? orc_rank_low_##S(A[xi], B, m) : m;                       \
    }                                                                                 \
    xbar[p] = m;                                                                      \
    for (int64_t j = 0; j < p; ++j) {                                                 \
        int64_t yj = orc_block_start(m, p, j);                                        \
        ybar[j] = (yj < m) ? orc_rank_high_##S(B[yj], A, n) : n;                      \
    }                                                                                 \
    ybar[p] = n;                                                                      \
}                                                                                     \
                                                                                      \
/* The paper's algorithm run on the host: Steps 1-4, then every one of the 2p   */  \
/* subproblems merged with the stable two-pointer merge.  table (6*2p int64)    */  \
/* receives the subproblems as orc_subproblems writes them.                     */  \
void orc_paper_merge_##S(const T* A, const uint32_t* Av, int64_t n,                   \
                         const T* B, const uint32_t* Bv, int64_t m, int64_t p,        \
                         T* C, uint32_t* Cv, int64_t* xbar, int64_t* ybar,            \
                         int64_t* table)                                              \
{                                                                                     \
    orc_cross_ranks_##S(A, n, B, m, p, xbar, ybar);                                   \
    orc_subproblems(n, m, p, xbar, ybar, table);                                      \
    for (int64_t k = 0; k < 2 * p; ++k) {                                             \
        const int64_t* row = table + 6 * k;                                           \
        int64_t c0 = row[4];                                                          \
        if (k < p)   /* A-side: own = A, other = B */                                 \
            orc_merge_two_pointer_##S(A + row[0], Av + row[0], row[1] - row[0],       \
                                      B + row[2], Bv + row[2], row[3] - row[2],       \
                                      C + c0, Cv + c0);                               \
        else         /* B-side: own = B, other = A; A still wins ties */              \
            orc_merge_two_pointer_##S(A + row[2], Av + row[2], row[3] - row[2],       \
                                      B + row[0], Bv + row[0], row[1] - row[0],       \
                                      C + c0, Cv + c0);                               \
    }                                                                                 \
}                                                                                     \
                                                                                      \
/* Many independent merges (Section 3: the merge applied to several pairs).     */  \
/* Pair k merges A[a_off[k]..a_off[k+1]) with B[b_off[k]..b_off[k+1]) into      */  \
/* C[a_off[k]+b_off[k] ..).  Offsets start at 0.                                */  \
void orc_merge_batched_##S(int64_t pairs,                                             \
                           const int64_t* a_off, const T* A, const uint32_t* Av,      \
                           const int64_t* b_off, const T* B, const uint32_t* Bv,      \
                           T* C, uint32_t* Cv)                                        \
{                                                                                     \
    for (int64_t k = 0; k < pairs; ++k) {                                             \
        int64_t a0 = a_off[k], a1 = a_off[k + 1], b0 = b_off[k], b1 = b_off[k + 1];   \
        orc_merge_two_pointer_##S(A + a0, Av + a0, a1 - a0, B + b0, Bv + b0, b1 - b0, \
                                  C + a0 + b0, Cv + a0 + b0);                         \
    }                                                                                 \
}                                                                                     \
                                                                                      \
/* Stable merge sort of Section 3: consecutive blocks of `run` elements are     */  \
/* sorted sequentially (stable insertion sort), then rounds merge adjacent      */  \
/* sorted runs pairwise; an unpaired last run is copied.  Input and output      */  \
/* alternate between (keys, vals) and (tk, tv); the result ends in keys/vals.   */  \
void orc_merge_sort_##S(T* keys, uint32_t* vals, int64_t n, int64_t run,              \
                        T* tk, uint32_t* tv)                                          \
{                                                                                     \
    if (run < 1) run = 1;                                                             \
    for (int64_t lo = 0; lo < n; lo += run) {                                         \
        int64_t hi = lo + run < n ? lo + run : n;                                     \
        for (int64_t a = lo + 1; a < hi; ++a) {                                       \
            T k = keys[a]; uint32_t v = vals[a];                                      \
            int64_t b = a;                                                            \
            while (b > lo && k < keys[b - 1]) {                                       \
                keys[b] = keys[b - 1]; vals[b] = vals[b - 1]; --b;                    \
            }                                                                         \
            keys[b] = k; vals[b] = v;                                                 \
        }                                                                             \
    }                                                                                 \
    T* sk = keys; uint32_t* sv = vals; T* dk = tk; uint32_t* dv = tv;                 \
    for (int64_t w = run; w < n; w *= 2) {                                            \
        for (int64_t lo = 0; lo < n; lo += 2 * w) {                                   \
            int64_t mid = lo + w < n ? lo + w : n;                                    \
            int64_t hi = lo + 2 * w < n ? lo + 2 * w : n;                             \
            orc_merge_two_pointer_##S(sk + lo, sv + lo, mid - lo, sk + mid, sv + mid, \
                                      hi - mid, dk + lo, dv + lo);                    \
        }                                                                             \
        T* t1 = sk; sk = dk; dk = t1;                                                 \
        uint32_t* t2 = sv; sv = dv; dv = t2;                                          \
    }                                                                                 \
    if (sk != keys) {                                                                 \
        memcpy(keys, sk, (size_t)n * sizeof(T));                                      \
        memcpy(vals, sv, (size_t)n * sizeof(uint32_t));                               \
    }                                                                                 \
}

DEFINE_ORACLE(u32, uint32_t)
DEFINE_ORACLE(i32, int32_t)
DEFINE_ORACLE(u64, uint64_t)
DEFINE_ORACLE(f32, float)
