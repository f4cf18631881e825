/*
 * tm.h -- C ABI of the GB300 (sm_103a) stable parallel merge library.
 *
 * The library implements the merge of Traeff, "Simplified, stable parallel
 * merging" (arXiv:1202.6575):
 *   Steps 1-2  (Section 2): cross ranks of the p block starts of A in B
 *              (rank_low) and of B in A (rank_high), by binary search;
 *   Steps 3-4  (Section 2): the 2p disjoint subproblems those ranks define
 *              (cases (a)-(e) and their B-side mirror), each merged stably;
 *   Section 3: the same merge applied to many pairs at once, and the stable
 *              merge sort built from it.
 * A learned cross-rank proposal (not in the paper) narrows the rank_high
 * searches of a large, repeatedly merged base array to a short window that
 * is verified against the definition of rank_high and replaced by the full
 * search when the check fails.
 *
 * Conventions for every entry point:
 *  - Key arrays are non-decreasing under the key type's order: TM_KEY_U32 and
 *    TM_KEY_U64 unsigned, TM_KEY_I32 signed, TM_KEY_F32 IEEE '<' (no NaN;
 *    -0.0 and +0.0 are equal keys).  Payloads are opaque 32-bit words that
 *    travel with their keys.  Arrays are structure-of-arrays.
 *  - Stability (Section 2): on equal keys every element of A precedes every
 *    element of B, and each side keeps its input order.  A and B are never
 *    exchanged.  The output is therefore unique.
 *  - All pointers named *_keys, *_vals, workspace, offsets, xbar, ybar,
 *    status and model are DEVICE pointers owned by the caller, except where
 *    a comment says "host".  Key pointers must be aligned to the key size,
 *    payload pointers to 4 bytes, workspace and model to 256 bytes.  Outputs
 *    must not overlap inputs.  The library allocates no device memory.
 *  - Every call is asynchronous on `stream` (NULL = the legacy default
 *    stream) and returns after enqueueing work.  Argument errors return
 *    TM_ERR_INVALID / TM_ERR_WORKSPACE / TM_ERR_UNSUPPORTED synchronously and
 *    launch nothing; a failed launch returns TM_ERR_CUDA.  Conditions that
 *    only the device can see (a subproblem larger than its staging buffer, a
 *    bounded wait that gave up) are written to a device status word that
 *    tm_read_status() returns; kernels never trap.
 *  - Payload width: payloads are 4-byte words unless cfg->payload_bytes = 8
 *    selects 8-byte words (tm_merge, tm_merge_tiles, tm_merge_batched,
 *    tm_merge_sort and the autotuners; the payload pointers keep their
 *    uint32_t* type and must then be 8-byte aligned).  tm_merge_noalloc and
 *    the learned calls take 4-byte payloads only.
 *  - Keys-only merges: every merge and sort call accepts NULL for all of its
 *    payload pointers (a_vals, b_vals and c_vals together; vals and tmp_vals
 *    together for the sort) and then moves keys only (half the bytes for
 *    4-byte keys).  A mix of NULL and non-NULL payload pointers is
 *    TM_ERR_INVALID; tm_merge_noalloc, and cfg->split = TM_SPLIT_BLOCKS,
 *    return TM_ERR_UNSUPPORTED for keys only.
 *  - A workspace (or model) belongs to one call at a time: calls that use the
 *    same workspace must be ordered on the GPU (one stream, or events);
 *    overlapping ones race on its status word, work-queue counter, barrier
 *    count and arrays.
 *  - Lengths are element counts (int64_t, >= 0).  Empty inputs are valid.
 */
#ifndef TM_H
#define TM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TM_API __attribute__((visibility("default")))
#else
#define TM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st* tm_stream_t;

typedef enum {
    TM_OK = 0,
    TM_ERR_INVALID = 1,      /* bad argument (NULL, negative length, misaligned pointer, ...) */
    TM_ERR_UNSUPPORTED = 2,  /* unknown key type or configuration outside the kernel's limits */
    TM_ERR_WORKSPACE = 3,    /* workspace NULL or smaller than the matching *_workspace_size() */
    TM_ERR_CUDA = 4,         /* a CUDA runtime call or launch failed */
    TM_ERR_TIMEOUT = 5,      /* device: a bounded wait gave up (set in the status word) */
    TM_ERR_BOUNDS = 6        /* device: a subproblem exceeded its staging capacity */
} tm_status;

typedef enum {
    TM_KEY_U32 = 0,
    TM_KEY_I32 = 1,
    TM_KEY_U64 = 2,
    TM_KEY_F32 = 3
} tm_key_type;

/* Tuning knobs.  A NULL tm_config*, or 0 in a field, selects the default. */
typedef struct tm_config {
    int64_t p;          /* blocks per input array (Section 2).  0: derived so that one
                           subproblem fits `tile` elements: p = ceil((n + m) / tile). */
    int32_t tile;       /* max elements (A piece + B piece) a CTA stages in shared memory;
                           default 2048 */
    int32_t threads;    /* consumer threads per CTA: 128 or 256 (512 with TM_SPLIT_BLOCKS);
                           default 128 */
    int32_t grid;       /* CTAs of the persistent kernels; default: resident CTAs per SM
                           x SM count */
    int32_t stages;     /* input stages of the persistent tile kernel: 2, 3 or 4 with
                           TM_SPLIT_DIAGONAL (default 4 when two CTAs fit on an SM, else 3,
                           else 2), 1, 2 or 4 with TM_SPLIT_BLOCKS (default 2) */
    int32_t split;      /* how a CTA divides its staged tile among its threads:
                           TM_SPLIT_DIAGONAL (2; also 0 = default) or TM_SPLIT_BLOCKS (1) */
    int32_t wait_ms;    /* limit of every wait of the persistent tile kernel on a stage
                           barrier, in milliseconds; default 2000.  When a wait gives up the
                           kernel sets TM_ERR_TIMEOUT in the status word and returns. */
    int32_t test_drop_tile; /* testing only (0 = off): each CTA of the persistent tile kernel
                           withholds the readiness signal of its test_drop_tile-th staged
                           tile, so its consumers' wait runs out (TM_ERR_TIMEOUT); the
                           merge result is then incomplete.  Exercises the bounded waits. */
    int32_t unfused;    /* tm_merge only: 1 forces the separate search, plan and merge
                           launches where the fused single launch would be used (below) */
    int32_t partition;  /* tm_merge only: TM_PARTITION_BLOCKS (0, the paper's method) or
                           TM_PARTITION_DIAGONALS (1, an ablation: equal output ranges) */
    int32_t payload_bytes; /* bytes of one payload word: 4 (also 0, the default) or 8; with 8
                           every payload pointer of the call points to 8-byte words (8-byte
                           aligned) although it is declared uint32_t* */
    int32_t trace;      /* tm_merge only, profiling (0 = off): 1 makes the fused single launch
                           record per-CTA phase timestamps in the workspace (which then needs
                           tm_merge_workspace_size with the same cfg); tm_merge_phase_times
                           reads them */
    int32_t merge_ways; /* tm_merge_sort only: runs merged per pass over memory, 2 (also 0, the
                           default: one pairwise round per pass) or 4 (two rounds per pass,
                           below) */
} tm_config;

/* How tm_merge divides the merge into subproblems.  TM_PARTITION_BLOCKS is
 * the paper's (Section 2): p blocks per input, cross ranks of the block
 * starts, the five cases.  TM_PARTITION_DIAGONALS, kept as an ablation, cuts
 * the output into equal ranges of `tile` elements instead (the equal-output
 * partitioning of prior work the paper discusses in Section 1): one search
 * per cut along its output diagonal (the co-rank i with B[d-i-1] < A[i] and
 * A[i-1] <= B[d-i]), then the same tile merge.  Same result. */
enum { TM_PARTITION_BLOCKS = 0, TM_PARTITION_DIAGONALS = 1 };

/* In-CTA split modes.  TM_SPLIT_BLOCKS applies the paper's rule again inside
 * the CTA: `threads` blocks per piece, rank_low of every A-block start in the
 * B piece, rank_high of every B-block start in the A piece, and the 2*threads
 * sub-subproblems of Steps 3-4, two per thread.  TM_SPLIT_DIAGONAL gives every
 * thread the same number of outputs: thread t starts at output t*ceil(L/threads)
 * of the tile, at the split the position formulas of Section 2 fix there
 * (i A elements before it: B[d-i-1] < A[i] and A[i-1] <= B[d-i]).  Both give
 * the identical (unique) stable merge.  A tile longer than 33 runs per thread
 * (tile > 33 * threads) uses TM_SPLIT_BLOCKS. */
enum { TM_SPLIT_BLOCKS = 1, TM_SPLIT_DIAGONAL = 2, TM_SPLIT_DEFAULT = TM_SPLIT_DIAGONAL };

/* Human-readable name of a status code (static storage). */
TM_API const char* tm_status_str(tm_status s);

/* Library version, for the binding's load check. */
TM_API int tm_version(void);

/* Name of the CUDA error behind the calling thread's most recent
 * TM_ERR_CUDA (a kernel launch or CUDA runtime call of this library that
 * failed: memset, copy, event, graph or stream call); "cudaSuccess" if none
 * was recorded.  Static storage. */
TM_API const char* tm_last_cuda_error(void);

/* ------------------------------------------------------------------------ */
/* Device status word                                                        */
/* ------------------------------------------------------------------------ */

/* Copies the 32-bit device status word at `status` (device) to the host after
 * synchronising `stream`.  Returns TM_OK when no kernel reported a problem,
 * otherwise the first device-side code (TM_ERR_BOUNDS, TM_ERR_TIMEOUT).
 * For tm_merge the status word is the first 4 bytes of its workspace; for the
 * batched and sort calls likewise. */
TM_API tm_status tm_read_status(const void* status, tm_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Single merge (Section 2, Steps 1-4)                                       */
/* ------------------------------------------------------------------------ */

/* The number of blocks p that tm_merge uses for (n, m, cfg) when payloads
 * are given (keys-only merges above the fused range may use fewer: see
 * tm_merge). */
TM_API int64_t tm_merge_blocks(int64_t n, int64_t m, const tm_config* cfg);

/* Workspace bytes tm_merge needs: a 256-byte control block (status word,
 * work-queue counter), the two cross-rank arrays xbar[0..p], ybar[0..p]
 * (int64) and the 2p tile records. */
TM_API size_t tm_merge_workspace_size(int64_t n, int64_t m, const tm_config* cfg);

/* Stable merge of A (n keys + payloads) and B (m) into C (n + m).
 * Steps 1-2 run as one search kernel (2p binary searches), the stream order
 * is the single synchronisation of Section 2, and Steps 3-4 run as a
 * planning kernel (one tile record per subproblem) and the persistent
 * staged tile-merge kernel.  Equivalent to tm_cross_ranks,
 * tm_plan_subproblems and tm_merge_tiles on the workspace's arrays.
 * Small merges (p <= 16384 and default in-CTA settings: no cfg->threads,
 * stages, grid, split other than the default, wait_ms or test_drop_tile)
 * run instead as one cooperative launch of the tile kernel: its warps do
 * the 2p searches (one warp per search, 32 probes per round), a grid-wide
 * barrier (bounded wait: TM_ERR_TIMEOUT) stands for the synchronisation,
 * and each CTA then selects the subproblems of its own processing elements
 * (Steps 3-4) and merges them; the result is identical.  cfg->unfused = 1
 * keeps the separate launches.  Above that range, with no cfg field set
 * but payload_bytes and merge_ways, keys-only merges (all payload pointers
 * NULL) use 8192-element tiles and 256 consumer threads, so fewer blocks
 * than tm_merge_blocks reports (the workspace size covers them), and merges
 * of 8-byte payloads use 256 consumer threads.
 * The control block (status word in its first 4 bytes) is cleared by this
 * call. */
TM_API tm_status tm_merge(tm_key_type kt,
                   const void* a_keys, const uint32_t* a_vals, int64_t n,
                   const void* b_keys, const uint32_t* b_vals, int64_t m,
                   void* c_keys, uint32_t* c_vals,
                   void* workspace, size_t workspace_bytes,
                   const tm_config* cfg, tm_stream_t stream);

/* Phase times of the last fused single launch of tm_merge made with
 * cfg->trace = 1 on this workspace (same n, m, cfg): synchronises `stream`,
 * reads the per-CTA %globaltimer stamps and writes to us_out (host, 6
 * doubles, microseconds): [0] Steps 1-2 searches (kernel entry of the first
 * CTA to the last CTA done searching), [1] the synchronisation after them
 * (grid barrier), [2] Steps 3-4 selection, [3] a second barrier (0 when the
 * launch has none), [4] the merges (to the last CTA's last store), [5] the
 * whole kernel.  TM_ERR_INVALID when the workspace holds no trace (the call
 * did not take the fused launch, or cfg->trace was 0). */
TM_API tm_status tm_merge_phase_times(const void* workspace, int64_t n, int64_t m, const tm_config* cfg,
                                      double* us_out, tm_stream_t stream);

/* The per-CTA stamps behind tm_merge_phase_times (same workspace, n, m,
 * cfg): synchronises `stream` and writes to out (host memory, room for
 * `capacity` words), for each CTA c of the last traced fused launch, 8
 * words out[8c .. 8c+7]: %globaltimer nanoseconds at kernel entry, searches
 * done, grid barrier passed, its own subproblems selected (twice: the
 * launch has no second barrier), merges done (its last store issued), its
 * first staged tile landed; then the number of tiles the CTA merged.
 * *ctas receives the CTA count, also when `capacity` is too small (then
 * TM_ERR_INVALID and nothing is written; out may be NULL with capacity 0
 * to ask for the count); otherwise the errors of tm_merge_phase_times. */
TM_API tm_status tm_merge_trace(const void* workspace, int64_t n, int64_t m, const tm_config* cfg,
                                uint64_t* out, int64_t capacity, int64_t* ctas, tm_stream_t stream);

/* Steps 1 and 2 alone (Section 2): xbar[i] = rank_low(A[x_i], B) for i < p,
 * xbar[p] = m; ybar[j] = rank_high(B[y_j], A) for j < p, ybar[p] = n, with
 * the block starts x_i, y_j of Section 2 (the first n mod p blocks one
 * longer).  The start of an empty block is the +inf sentinel, so its cross
 * rank is the other array's length.  xbar and ybar hold p + 1 int64 each. */
TM_API tm_status tm_cross_ranks(tm_key_type kt,
                         const void* a_keys, int64_t n,
                         const void* b_keys, int64_t m, int64_t p,
                         int64_t* xbar, int64_t* ybar, tm_stream_t stream);

/* Steps 3 and 4, first half (subproblem selection): for each of the 2p
 * processing elements of tm_cross_ranks' (A, B, p) whose block is not empty,
 * one tile record of tm_tile_record_bytes() bytes (device, 16-byte aligned):
 * the subproblem's A range, B range and output offset, chosen by the five
 * cases (a)-(e) of Step 3 and their mirror in Step 4.  Records are stored
 * in merge-path order (by output offset), tm_plan_tile_count(n, m, p) of
 * them; `tiles` must hold 2p records.  Layout of a record (48 bytes):
 * int64 a0, b0, c0 (first A index, first B index, first output index),
 * int32 nA, nB, int32 first (1 on a merge's first record), padding. */
TM_API size_t tm_tile_record_bytes(void);
TM_API int64_t tm_plan_tile_count(int64_t n, int64_t m, int64_t p);
TM_API tm_status tm_plan_subproblems(int64_t n, int64_t m, int64_t p,
                                     const int64_t* xbar, const int64_t* ybar,
                                     void* tiles, const tm_config* cfg, tm_stream_t stream);

/* Largest subproblem of (n, m, p): ceil(n/p) + ceil(m/p) elements (each
 * range lies inside one block of its array).  -1 on bad arguments. */
TM_API int32_t tm_merge_tile_cap(int64_t n, int64_t m, int64_t p);

/* Steps 3 and 4, second half (the stable merges): merges every tile record
 * into C with the persistent staged tile-merge kernel.  Consecutive records
 * (adjacent on the merge path) are packed into one staged tile while the
 * total stays within `cap`, which must bound every single record
 * (tm_merge_tile_cap).  `control` is a 256-byte device block: int32 status
 * word at byte 0 (set on a device-side error, not cleared here), work-queue
 * counter at byte 8 (reset by this call). */
TM_API tm_status tm_merge_tiles(tm_key_type kt,
                                const void* a_keys, const uint32_t* a_vals, int64_t n,
                                const void* b_keys, const uint32_t* b_vals, int64_t m,
                                const void* tiles, int64_t n_tiles, int32_t cap,
                                void* c_keys, uint32_t* c_vals, void* control,
                                const tm_config* cfg, tm_stream_t stream);

/* The subproblems of Steps 3-4 as the device computes them: for k < p the
 * A-side processing element k, for k >= p the B-side one (k - p).  Row k of
 * `table` (device, 2p x 4 int64) receives a0, a1, b0, b1: the half-open A and
 * B ranges of the subproblem; its output starts at C[a0 + b0].  Used to check
 * the device's reading of the five cases against the paper's worked example
 * and the host oracle. */
TM_API tm_status tm_subproblems(int64_t n, int64_t m, int64_t p,
                                const int64_t* xbar, const int64_t* ybar,
                                int64_t* table, tm_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Many merges at once and the stable merge sort (Section 3)                 */
/* ------------------------------------------------------------------------ */

/* Workspace bytes of tm_merge_batched for (num_pairs, total_a, total_b, cfg). */
TM_API size_t tm_merge_batched_workspace_size(int64_t num_pairs, int64_t total_a, int64_t total_b,
                                              const tm_config* cfg);

/* num_pairs independent stable merges.  Pair k merges A[a_offsets[k] ..
 * a_offsets[k+1]) with B[b_offsets[k] .. b_offsets[k+1]) into C from
 * a_offsets[k] + b_offsets[k] (CSR offsets, device int64, num_pairs + 1
 * each, starting at 0 and ending at total_a / total_b).  Each pair is merged
 * by the paper's method with its own block count p_k = ceil((n_k + m_k) /
 * tile): one search kernel and one planning kernel cover all pairs, then one
 * persistent tile-merge launch pulls every pair's subproblems from a device
 * work queue.  No host synchronisation: the call can be captured in a CUDA
 * graph (tm_graph_capture_begin/end).  cfg NULL uses the configuration the
 * autotuner chose for this key type and size, if any, else the defaults.
 * The status word is the first 4 bytes of the workspace. */
TM_API tm_status tm_merge_batched(tm_key_type kt, int64_t num_pairs,
                                  const int64_t* a_offsets, const void* a_keys, const uint32_t* a_vals,
                                  int64_t total_a,
                                  const int64_t* b_offsets, const void* b_keys, const uint32_t* b_vals,
                                  int64_t total_b,
                                  void* c_keys, uint32_t* c_vals, void* workspace, size_t workspace_bytes,
                                  const tm_config* cfg, tm_stream_t stream);

/* Workspace bytes of tm_merge_sort for n elements. */
TM_API size_t tm_merge_sort_workspace_size(int64_t n, const tm_config* cfg);

/* Stable sort of (keys, vals) by key (Section 3): consecutive runs of 4096
 * elements are sorted inside one CTA each (a stable LSD radix sort of the
 * keys' order-preserving images, 8 bits per pass, skipping the bytes in
 * which all keys of the run agree), then ceil(log2(n / 4096)) rounds merge
 * adjacent runs pairwise (an unpaired last run is copied), every round one
 * batched merge of uniform pairs.  With
 * cfg->merge_ways = 4, two consecutive rounds are done in one pass over
 * memory: groups of four runs R0..R3 become merge(merge(R0, R1), merge(R2,
 * R3)), the subproblems chosen by the paper's method on the outer merge of
 * the two intermediate sequences (which stay in shared memory); a last odd
 * round is pairwise (pairwise rounds are also taken with cfg->split =
 * TM_SPLIT_BLOCKS and tiles above 4606).  Passes alternate between (keys,
 * vals) and (tmp_keys, tmp_vals); the result ends in (keys, vals).  Equal
 * keys keep their input order.  Other values of merge_ways return
 * TM_ERR_UNSUPPORTED. */
TM_API tm_status tm_merge_sort(tm_key_type kt, void* keys, uint32_t* vals, int64_t n,
                               void* tmp_keys, uint32_t* tmp_vals, void* workspace, size_t workspace_bytes,
                               const tm_config* cfg, tm_stream_t stream);

/* Segmented stable sort: num_segments independent segments of one array,
 * segment q = (keys, vals)[seg_offsets[q], seg_offsets[q+1]), each sorted
 * stably by key (Section 3's merge sort inside every segment: runs of at
 * most 4096 elements that never cross a segment boundary, then rounds that
 * merge each segment's neighbouring runs pairwise, one batched merge per
 * round; a segment already sorted is copied).  seg_offsets is HOST memory
 * (num_segments + 1 int64, from 0, non-decreasing, ending at n): the host
 * counts runs and pairs per round, the offsets are copied into the
 * workspace from pageable host memory (so this call is not
 * graph-capturable) and device kernels write the run and pair descriptors.
 * Invalid offsets return TM_ERR_INVALID.  Passes alternate between (keys,
 * vals) and (tmp_keys, tmp_vals); the result ends in (keys, vals).  The
 * paper treats one array; independent segments are this library's. */
TM_API size_t tm_merge_sort_segmented_workspace_size(int64_t n, const int64_t* seg_offsets, int64_t num_segments,
                                                     const tm_config* cfg);
TM_API tm_status tm_merge_sort_segmented(tm_key_type kt, void* keys, uint32_t* vals, int64_t n,
                                         const int64_t* seg_offsets, int64_t num_segments, void* tmp_keys,
                                         uint32_t* tmp_vals, void* workspace, size_t workspace_bytes,
                                         const tm_config* cfg, tm_stream_t stream);

/* Autotuner (not in the paper): runs tm_merge_batched (resp. tm_merge_sort on
 * a fresh device copy of src into keys/vals per trial) once per candidate
 * configuration -- tile {1024, 2048, 4096} x threads {128, 256} x stages
 * {3, 4}, diagonal in-CTA split, skipping those whose workspace exceeds
 * workspace_bytes -- timed with CUDA events on `stream`, and keeps the
 * fastest for later calls with cfg NULL (or setting only payload_bytes) on
 * the same key type, payload width and size (power-of-two bucket of the
 * element count).  Synchronises the stream.  On input best->payload_bytes (0
 * or 4: 4-byte payloads, 8: 8-byte payloads; best NULL: 4) selects the
 * payload width of the trials; on return *best holds the chosen
 * configuration. */
TM_API tm_status tm_autotune_batched(tm_key_type kt, int64_t num_pairs,
                                     const int64_t* a_offsets, const void* a_keys, const uint32_t* a_vals,
                                     int64_t total_a,
                                     const int64_t* b_offsets, const void* b_keys, const uint32_t* b_vals,
                                     int64_t total_b,
                                     void* c_keys, uint32_t* c_vals, void* workspace, size_t workspace_bytes,
                                     tm_config* best, tm_stream_t stream);
TM_API tm_status tm_autotune_sort(tm_key_type kt, const void* src_keys, const uint32_t* src_vals, int64_t n,
                                  void* keys, uint32_t* vals, void* tmp_keys, uint32_t* tmp_vals,
                                  void* workspace, size_t workspace_bytes, tm_config* best,
                                  tm_stream_t stream);
/* Forgets every autotuned configuration; returns how many there were. */
TM_API int tm_autotune_clear(void);

/* ------------------------------------------------------------------------ */
/* CUDA graphs                                                               */
/* ------------------------------------------------------------------------ */

/* Capture every call issued on `stream` (not the legacy NULL stream) between
 * begin and end into a CUDA graph (thread-local capture mode); replay it
 * with tm_graph_launch on any stream.  The replay reuses the pointers and
 * sizes of the captured calls.  tm_graph_end returns TM_ERR_CUDA if the
 * capture failed (e.g. a call synchronised the stream, or a graph was
 * destroyed on this thread meanwhile).  Make each kind of call once
 * outside a capture first: the first call of a kernel configuration sets
 * its shared-memory limit, which a capture should not have to do. */
typedef struct tm_graph tm_graph;
TM_API tm_status tm_graph_capture_begin(tm_stream_t stream);
TM_API tm_status tm_graph_capture_end(tm_stream_t stream, tm_graph** out);
TM_API tm_status tm_graph_launch(tm_graph* g, tm_stream_t stream);
TM_API void tm_graph_destroy(tm_graph* g);

/* ------------------------------------------------------------------------ */
/* Learned cross-rank proposal (not in the paper)                            */
/* ------------------------------------------------------------------------ */

/* A model of the distribution of a large sorted float32 base array X that is
 * merged again and again with incoming sorted batches (base' = merge(base,
 * batch), base on the A side so that older keys win ties).  It proposes the
 * cross ranks of Steps 1-2; every proposal is searched only in a window and
 * then checked against the definition of rank_low / rank_high (Section 2);
 * a failed check runs the full binary search, so results never depend on
 * the model.
 *
 * Model: S segments with knot keys K[s] = X[floor(s N / S)] (K[S] = X[N-1])
 * and their ranks R[s] in the current base (a piecewise-linear CDF), plus a
 * two-layer MLP (2 inputs, H ReLU units, 1 output) that predicts the
 * residual of the piecewise-linear rank in units of the segment's size, from
 * the key's position t in its segment and the segment index.  The error
 * bound eps (calibrated, in segment units) sets the search window.  Training
 * is full-batch Adam on (key, exact rank_high) pairs.
 *
 * Memory: one caller-owned device buffer of tm_cdf_model_bytes(S, H) bytes
 * (256-byte aligned).  Layout, little endian: a 256-byte header
 *   int32 S; int32 H; float eps; int32 cur; int64 N; uint64 fallbacks;
 *   uint64 learned_searches; int64 adam_steps; float loss; uint32 arrived
 *   (a completion counter of tm_cross_ranks_learned, zero between calls);
 * then, each section starting on a 256-byte boundary: float K[S+1];
 * int64 R0[S+1]; int64 R1[S+1] (R_cur is R0 when cur = 0); float params[4H+1]
 * = W1 (H x 2, row major), b1 (H), w2 (H), b2; float adam_m[4H+1];
 * float adam_v[4H+1]; float grad[4H+1]; float eps_seg[S] (per-segment error
 * bound, 0 for a segment without labels).  Every call takes the model's S
 * and H; none reads the header back, so all of them can be graph-captured. */
enum { TM_LEARNED_ADVANCE = 1 };

TM_API size_t tm_cdf_model_bytes(int segments, int hidden);

/* Knots from the base (n sorted keys), parameters from init_params (device,
 * 4H+1 floats), Adam state zeroed, N = n. */
TM_API tm_status tm_cdf_init(void* model, int segments, int hidden, const float* base_keys, int64_t n,
                             const float* init_params, tm_stream_t stream);

/* Gradient (device, 4H+1 floats) and loss (device float) of the mean
 * 0.5 * (y - tau)^2 over `count` labelled keys, at the current parameters;
 * no update.  labels: exact rank_high of q in the base (int64). */
TM_API tm_status tm_cdf_grad(void* model, int segments, int hidden, const float* q, const int64_t* labels,
                             int64_t count, float* grad_out, float* loss_out, tm_stream_t stream);

/* `steps` full-batch Adam steps (beta 0.9 / 0.999, eps 1e-8, learning rate
 * lr) on the labelled keys: one forward+backward kernel and one update
 * kernel per step. */
TM_API tm_status tm_cdf_train(void* model, int segments, int hidden, const float* q, const int64_t* labels,
                              int64_t count, int steps, float lr, tm_stream_t stream);

/* Predicted rank (float) of every key. */
TM_API tm_status tm_cdf_predict(const void* model, int segments, int hidden, const float* q, int64_t count,
                                float* pred, tm_stream_t stream);

/* eps = max |y - tau| over the labelled keys (segment units), and per
 * segment the same maximum over the labels falling in it. */
TM_API tm_status tm_cdf_calibrate(void* model, int segments, int hidden, const float* q, const int64_t* labels,
                                  int64_t count, tm_stream_t stream);

/* Steps 1-2 with learned proposals: A = the model's current base (n keys),
 * B = a batch (m keys), p blocks; same results as tm_cross_ranks.  The
 * B-block starts, which search the large base, use the model: each searches
 * the base within 3 eps_s * (segment size) + 32 ranks of the proposal (eps_s
 * the calibrated error of the key's segment, the global one when the
 * segment had no labels), and the answer is verified.  The A-block starts
 * search the small batch by plain bisection.  With TM_LEARNED_ADVANCE in
 * flags the knot ranks of merge(A, B) are written to the other rank buffer
 * (R'[s] = R[s] + rank_low(K[s], B)) and made current, and N becomes n + m:
 * the model then describes the merged base (the launch's last CTA to finish
 * flips the buffers, so calls on one model must not overlap on the GPU).
 * Counts of learned searches and of fallbacks accumulate in the header.
 * Inside the window the probes are placed from the data (the proposal, the
 * segment's density, then interpolation between probed keys); bisection
 * finishes.  The result never depends on where the probes fall. */
TM_API tm_status tm_cross_ranks_learned(void* model, int segments, int hidden, const float* a_keys, int64_t n,
                                        const float* b_keys, int64_t m, int64_t p, int64_t* xbar, int64_t* ybar,
                                        int flags, tm_stream_t stream);

/* tm_merge for float keys with the learned Steps 1-2 (same workspace as
 * tm_merge; same result). */
TM_API tm_status tm_merge_learned(void* model, int segments, int hidden,
                                  const float* a_keys, const uint32_t* a_vals, int64_t n,
                                  const float* b_keys, const uint32_t* b_vals, int64_t m,
                                  float* c_keys, uint32_t* c_vals, void* workspace, size_t workspace_bytes,
                                  const tm_config* cfg, int flags, tm_stream_t stream);

/* Stable merge that allocates nothing and needs no workspace.  The paper has
 * no counterpart; this is a convenience of the library.  It exists for
 * callers that cannot call cudaMalloc or hand the library a workspace: code
 * hosted by a framework that passes it only its input and output buffers,
 * loops that must never hit the allocator (an allocation can block or
 * synchronise the device), or processes whose device memory is fully
 * reserved.  The computation and the result are those of tm_merge.
 *
 * The cross ranks live in one file-scope device array inside the library,
 * 4 MiB, which every GPU that loads the library keeps until the process
 * exits.  It holds p + 1 <= 262144 entries per side, so (n, m, cfg) must give
 * tm_merge_blocks() <= 262143 (about 2^29 elements at the default tile);
 * larger requests return TM_ERR_WORKSPACE and launch nothing.
 * The first call on each device looks the array's device address up once
 * (cudaGetSymbolAddress), and again after the device's context changes
 * (cudaDeviceReset); make that first call before any stream capture.
 * All calls share the one array and it keeps the last call's contents: two
 * calls that overlap on the GPU (other streams, other host threads) race and
 * corrupt each other's result, so keep calls ordered on one stream.
 * `status` (device int32, may be NULL) is an output: the call clears it and
 * a kernel sets it on a device-side error, as the status word of tm_merge.
 * Of tm_config it reads p, tile and threads (128, 256 or 512); it always
 * merges with one CTA per subproblem, so split, stages, grid and unfused do
 * not apply, and partition must be TM_PARTITION_BLOCKS (anything else, and a
 * thread count tm_merge refuses, returns TM_ERR_UNSUPPORTED). */
TM_API tm_status tm_merge_noalloc(tm_key_type kt,
                                  const void* a_keys, const uint32_t* a_vals, int64_t n,
                                  const void* b_keys, const uint32_t* b_vals, int64_t m,
                                  void* c_keys, uint32_t* c_vals, int32_t* status,
                                  const tm_config* cfg, tm_stream_t stream);

/* Batched rank search: out[k] = rank_low(q[k], X) (kind 0) or
 * rank_high(q[k], X) (kind 1) for k < count, by binary search (Section 2's
 * definitions).  q need not be sorted. */
TM_API tm_status tm_rank_search(tm_key_type kt, int kind,
                         const void* q, int64_t count,
                         const void* x_keys, int64_t len,
                         int64_t* out, tm_stream_t stream);

#ifdef __cplusplus
}  /* extern "C" */
#endif

#endif /* TM_H */
