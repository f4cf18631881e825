/*
 * CPU baseline: the paper's algorithm on the host's cores (Traeff,
 * "Simplified, stable parallel merging", Section 2), with one POSIX thread
 * per processing element as on the shared-memory machines the paper
 * targets.
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY.  The benchmark times it next to
 * the single-threaded oracle as a second CPU baseline, and the tests check
 * it against the oracle.  It shares nothing with the CUDA library.
 *
 * Thread t is processing element t (and t + T, t + 2T, ... when p exceeds
 * the thread count T): Steps 1-2 (its cross ranks xbar_t, ybar_t, by the
 * oracle's binary searches), the single synchronisation of Section 2 (the
 * threads of the search phase are joined), then Steps 3-4 (its A-side and
 * B-side subproblems by the five cases, the oracle's orc_subproblem) and
 * their stable two-pointer merges into C.
 */
#define _POSIX_C_SOURCE 200809L
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

int64_t orc_block_start(int64_t len, int64_t p, int64_t i);
void orc_subproblem(int64_t n, int64_t m, int64_t p, int64_t k, const int64_t* xbar, const int64_t* ybar,
                    int64_t* row);

#define DEFINE_PARALLEL(S, T)                                                                      \
int64_t orc_rank_low_##S(T x, const T* X, int64_t len);                                            \
int64_t orc_rank_high_##S(T x, const T* X, int64_t len);                                           \
void orc_merge_two_pointer_##S(const T* A, const uint32_t* Av, int64_t n, const T* B,              \
                               const uint32_t* Bv, int64_t m, T* C, uint32_t* Cv);                 \
                                                                                                   \
typedef struct {                                                                                   \
    const T* A; const uint32_t* Av; int64_t n;                                                     \
    const T* B; const uint32_t* Bv; int64_t m;                                                     \
    int64_t p, threads, t;                                                                         \
    T* C; uint32_t* Cv; int64_t* xbar; int64_t* ybar;                                              \
} par_job_##S;                                                                                     \
                                                                                                   \
static void* par_search_##S(void* arg)                      /* Steps 1-2 of PEs t, t + T, ... */   \
{                                                                                                  \
    par_job_##S* g = (par_job_##S*)arg;                                                            \
    const int64_t n = g->n, m = g->m, p = g->p;                                                    \
    for (int64_t i = g->t; i < p; i += g->threads) {                                               \
        int64_t xi = orc_block_start(n, p, i), yi = orc_block_start(m, p, i);                      \
        g->xbar[i] = (xi < n) ? orc_rank_low_##S(g->A[xi], g->B, m) : m;                           \
        g->ybar[i] = (yi < m) ? orc_rank_high_##S(g->B[yi], g->A, n) : n;                          \
    }                                                                                              \
    return NULL;                                                                                   \
}                                                                                                  \
                                                                                                   \
static void* par_merge_##S(void* arg)                       /* Steps 3-4 of PEs t, t + T, ... */   \
{                                                                                                  \
    par_job_##S* g = (par_job_##S*)arg;                                                            \
    const int64_t n = g->n, m = g->m, p = g->p;                                                    \
    for (int64_t k = g->t; k < 2 * p; k += g->threads) {                                           \
        int64_t row[6];                                                                            \
        orc_subproblem(n, m, p, k, g->xbar, g->ybar, row);                                         \
        if (k < p)                                                                                 \
            orc_merge_two_pointer_##S(g->A + row[0], g->Av + row[0], row[1] - row[0],              \
                                      g->B + row[2], g->Bv + row[2], row[3] - row[2],              \
                                      g->C + row[4], g->Cv + row[4]);                              \
        else                                                                                       \
            orc_merge_two_pointer_##S(g->A + row[2], g->Av + row[2], row[3] - row[2],              \
                                      g->B + row[0], g->Bv + row[0], row[1] - row[0],              \
                                      g->C + row[4], g->Cv + row[4]);                              \
    }                                                                                              \
    return NULL;                                                                                   \
}                                                                                                  \
                                                                                                   \
/* One fork-join phase; a thread that cannot be started runs in the caller. */                    \
static void par_phase_##S(void* (*fn)(void*), par_job_##S* jobs, pthread_t* tids, int* started,    \
                          int64_t threads)                                                         \
{                                                                                                  \
    for (int64_t t = 1; t < threads; ++t)                                                          \
        started[t] = pthread_create(&tids[t], NULL, fn, &jobs[t]) == 0;                            \
    fn(&jobs[0]);                                                                                  \
    for (int64_t t = 1; t < threads; ++t) {                                                        \
        if (started[t]) pthread_join(tids[t], NULL);                                               \
        else fn(&jobs[t]);                                                                         \
    }                                                                                              \
}                                                                                                  \
                                                                                                   \
/* Returns 0, or -1 when memory for the thread table is missing (nothing done). */                \
int orc_paper_merge_parallel_##S(const T* A, const uint32_t* Av, int64_t n,                        \
                                 const T* B, const uint32_t* Bv, int64_t m, int64_t p,             \
                                 int64_t threads, T* C, uint32_t* Cv, int64_t* xbar, int64_t* ybar) \
{                                                                                                  \
    if (threads < 1) threads = 1;                                                                  \
    if (threads > p) threads = p;                                                                  \
    par_job_##S* jobs = (par_job_##S*)malloc(sizeof(par_job_##S) * (size_t)threads);               \
    pthread_t* tids = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);                     \
    int* started = (int*)calloc((size_t)threads, sizeof(int));                                     \
    if (!jobs || !tids || !started) { free(jobs); free(tids); free(started); return -1; }          \
    for (int64_t t = 0; t < threads; ++t) {                                                        \
        par_job_##S j = {A, Av, n, B, Bv, m, p, threads, t, C, Cv, xbar, ybar};                    \
        jobs[t] = j;                                                                               \
    }                                                                                              \
    par_phase_##S(par_search_##S, jobs, tids, started, threads);                                   \
    xbar[p] = m;                                                                                   \
    ybar[p] = n;                                                                                   \
    par_phase_##S(par_merge_##S, jobs, tids, started, threads);  /* after the synchronisation */   \
    free(jobs);                                                                                    \
    free(tids);                                                                                    \
    free(started);                                                                                 \
    return 0;                                                                                      \
}

DEFINE_PARALLEL(u32, uint32_t)
DEFINE_PARALLEL(i32, int32_t)
DEFINE_PARALLEL(u64, uint64_t)
DEFINE_PARALLEL(f32, float)
