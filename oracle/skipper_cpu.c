/*
 * oracle/skipper_cpu.c -- TEST AND BENCHMARK INFRASTRUCTURE ONLY.
 *
 * Skipper (Algorithm 1) on host threads, the paper's own setting (Section IV,
 * Section VI-D), as a CPU baseline for the CUDA library: it is neither the
 * oracle nor a fallback of the library, and its results are checked with the
 * oracle's checker.  It measures what Section VI-D measures on the host:
 * parallelization gain (SGMM time over Skipper time on T threads, Fig. 10)
 * and serial slowdown (Skipper on one thread over SGMM, Fig. 11).
 *
 * What it computes, following Algorithm 1 and Section IV-C:
 *   * one state byte per vertex, ACC = 0, RSVD = 1, MCHD = 2 (lines 2-4);
 *   * every stored entry (x, y) of the CSR is an edge e(x, y) (line 5); loops
 *     are skipped (lines 6-7); u = min(x, y), v = max(x, y) (lines 8-9);
 *   * while neither u nor v is MCHD (line 10): CAS u ACC -> RSVD, and on
 *     failure test line 10 again (lines 11-12); holding u, while v is not
 *     MCHD, CAS v ACC -> MCHD; on success u := MCHD and the edge is a match
 *     (lines 13-16); if u is not MCHD afterwards it is released to ACC
 *     (lines 17-18).  u is held exclusively while RSVD, so lines 15 and 18
 *     are plain (release) stores.
 *   * scheduling (Section IV-C: contiguous blocks per thread, with stealing):
 *     rows [r0, r1) are cut into blocks of consecutive vertices holding about
 *     `block_edges` entries each; thread t owns the t-th contiguous run of
 *     blocks and walks it in order; a thread whose run is done steals blocks
 *     from the runs of the others.
 *   * matches are written as mate[u] = v, mate[v] = u by the thread that
 *     makes them (the library's output form) instead of per-thread buffers.
 *   * row_skip = 1 adds one test per entry that is not in Algorithm 1: once
 *     the row vertex x is MCHD the rest of row x is left (what SGMM does in
 *     CSR order and what the CUDA sweep does).  row_skip = 0 is Algorithm 1
 *     as printed: every entry is read and tested at line 10.
 *
 * With one thread and rows in order this is SGMM in CSR order (a pin in
 * tests/test_oracle_cpu_skipper.py).  Waits are bounded (a bad state would
 * otherwise spin forever): past the bound the call returns -2.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#define CPU_NONE 0xFFFFFFFFu
#define ACC 0
#define RSVD 1
#define MCHD 2
#define SPIN_LIMIT (1ull << 34)

typedef struct {
    int64_t begin, end;  /* blocks [begin, end) of this thread's run */
    int64_t next;        /* next block to take (atomic) */
    char pad[64];
} run_t;

typedef struct {
    const int64_t *offsets;
    const uint32_t *nbrs;
    uint64_t n;
    unsigned char *state;
    uint32_t *mate;
    const int64_t *block_row;  /* first row of each block, [nblocks + 1] */
    run_t *runs;
    int threads;
    int row_skip;
    int failed;                /* atomic: a wait ran past its bound */
    uint64_t *conflicts;       /* per thread: failed CAS at lines 11 and 14 */
} job_t;

typedef struct {
    job_t *job;
    int t;
} arg_t;

static unsigned char ld(unsigned char *p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }

static int cas(unsigned char *p, unsigned char expect, unsigned char desired)
{
    return __atomic_compare_exchange_n(p, &expect, desired, 0, __ATOMIC_ACQ_REL, __ATOMIC_ACQUIRE);
}

/* Algorithm 1, lines 6-18, for the edge (x, y).  Returns 0, or -1 when a wait
 * ran past SPIN_LIMIT. */
static int process_edge(job_t *J, uint64_t x, uint64_t y, uint64_t *cnf)
{
    if (x == y) return 0;
    uint64_t u = x < y ? x : y, v = x < y ? y : x;
    unsigned char *su = J->state + u, *sv = J->state + v;
    uint64_t spins = 0;
    while (ld(su) != MCHD && ld(sv) != MCHD) {
        if (!cas(su, ACC, RSVD)) {
            ++*cnf;
            if (++spins > SPIN_LIMIT) return -1;
            continue;
        }
        while (ld(sv) != MCHD) {
            if (cas(sv, ACC, MCHD)) {
                __atomic_store_n(su, MCHD, __ATOMIC_RELEASE);
                J->mate[u] = (uint32_t)v;
                J->mate[v] = (uint32_t)u;
                break;
            }
            ++*cnf;
            if (++spins > SPIN_LIMIT) {
                __atomic_store_n(su, ACC, __ATOMIC_RELEASE);
                return -1;
            }
        }
        if (ld(su) != MCHD) __atomic_store_n(su, ACC, __ATOMIC_RELEASE);
    }
    return 0;
}

static int run_block(job_t *J, int64_t b, uint64_t *cnf)
{
    for (int64_t x = J->block_row[b]; x < J->block_row[b + 1]; ++x) {
        for (int64_t i = J->offsets[x]; i < J->offsets[x + 1]; ++i) {
            if (J->row_skip && ld(J->state + x) == MCHD) break;
            if (process_edge(J, (uint64_t)x, J->nbrs[i], cnf)) return -1;
        }
    }
    return 0;
}

static void *worker(void *p)
{
    arg_t *a = (arg_t *)p;
    job_t *J = a->job;
    uint64_t cnf = 0;
    for (int k = 0; k < J->threads; ++k) {      /* own run first, then steal */
        run_t *r = J->runs + (a->t + k) % J->threads;
        for (;;) {
            int64_t b = __atomic_fetch_add(&r->next, 1, __ATOMIC_RELAXED);
            if (b >= r->end) break;
            if (run_block(J, b, &cnf)) {
                __atomic_store_n(&J->failed, 1, __ATOMIC_RELAXED);
                J->conflicts[a->t] = cnf;
                return NULL;
            }
            if (__atomic_load_n(&J->failed, __ATOMIC_RELAXED)) break;
        }
    }
    J->conflicts[a->t] = cnf;
    return NULL;
}

static double now_s(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

/* Skipper over rows [r0, r1) of the CSR with `threads` threads.  mate[n] is
 * set to CPU_NONE first (not timed) and receives the matches; *seconds is the
 * time of the parallel pass (state init included, as in Algorithm 1).
 * Returns the number of conflicts (failed CAS), -1 on allocation or thread
 * failure, -2 when a wait ran past its bound. */
int64_t cpu_skipper(uint64_t n, const int64_t *offsets, const uint32_t *nbrs, uint64_t r0,
                    uint64_t r1, int threads, uint64_t block_edges, int row_skip,
                    uint32_t *mate, double *seconds)
{
    if (threads < 1 || r1 > n || r0 > r1) return -1;
    if (block_edges == 0) block_edges = 1;
    for (uint64_t v = 0; v < n; ++v) mate[v] = CPU_NONE;
    /* blocks of consecutive rows with about block_edges entries each */
    uint64_t entries = (uint64_t)(offsets[r1] - offsets[r0]);
    uint64_t cap = (entries + (r1 - r0)) / block_edges + 2;
    int64_t *block_row = (int64_t *)malloc((cap + 1) * sizeof(int64_t));
    unsigned char *state = (unsigned char *)malloc(n ? n : 1);
    run_t *runs = (run_t *)calloc((size_t)threads, sizeof(run_t));
    uint64_t *conflicts = (uint64_t *)calloc((size_t)threads, sizeof(uint64_t));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    arg_t *args = (arg_t *)calloc((size_t)threads, sizeof(arg_t));
    if (!block_row || !state || !runs || !conflicts || !tid || !args) {
        free(block_row); free(state); free(runs); free(conflicts); free(tid); free(args);
        return -1;
    }
    int64_t nb = 0;
    block_row[nb++] = (int64_t)r0;
    uint64_t acc = 0;
    for (uint64_t x = r0; x < r1; ++x) {
        acc += (uint64_t)(offsets[x + 1] - offsets[x]) + 1;
        if (acc >= block_edges && x + 1 < r1 && (uint64_t)nb < cap) {
            block_row[nb++] = (int64_t)(x + 1);
            acc = 0;
        }
    }
    block_row[nb] = (int64_t)r1;
    for (int t = 0; t < threads; ++t) {
        runs[t].begin = runs[t].next = nb * t / threads;
        runs[t].end = nb * (t + 1) / threads;
    }
    job_t J = {offsets, nbrs, n, state, mate, block_row, runs, threads, row_skip, 0, conflicts};

    double t0 = now_s();
    memset(state, ACC, n ? n : 1);                       /* lines 3-4 */
    int started = 0, ok = 1;
    for (int t = 0; t < threads; ++t) {
        args[t].job = &J;
        args[t].t = t;
        if (pthread_create(tid + t, NULL, worker, args + t) != 0) { ok = 0; break; }
        ++started;
    }
    if (!ok) __atomic_store_n(&J.failed, 1, __ATOMIC_RELAXED);
    for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    *seconds = now_s() - t0;

    int64_t total = 0;
    for (int t = 0; t < threads; ++t) total += (int64_t)conflicts[t];
    int failed = J.failed;
    free(block_row); free(state); free(runs); free(conflicts); free(tid); free(args);
    if (!ok) return -1;
    if (failed) return -2;
    return total;
}
