/*
 * oracle/sgmm.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Sequential Greedy Maximal Matching (SGMM) over a CSR graph, as the paper
 * defines it in Section II-B (its maximal-matching background): one thread walks the
 * edges; an edge whose two endpoints are both unmarked is taken, and both
 * endpoints are marked.  In CSR order, once the source vertex of a row is
 * marked the rest of that row cannot yield a match, so the row is left
 * (Section II-B, the paragraph on CSR processing; Fig. 1 walks this on the
 * 4-vertex example).  Self-loops are never taken (Alg. 1 skips them).
 *
 * This file is the reference against which the CUDA path is checked.  It
 * shares no code, header or constant with the CUDA library.  Only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline leg may call it.
 *
 * Edge order (a reading; the paper fixes no order beyond walking the edges): rows
 * in ascending vertex id, neighbours in stored order; the first unmarked
 * neighbour wins.
 *
 * Output: mate[v] = partner of v, or 0xFFFFFFFF when v is unmatched (the
 * paper pads invalid match slots with -1, Section IV-C; the per-vertex mate
 * array is this library's output form).  pairs (optional) receives the taken
 * edges (min, max) in the order SGMM takes them.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#define ORACLE_NONE 0xFFFFFFFFu

/* Returns the number of matched pairs, or -1 on allocation failure or a
 * neighbour id outside [0, n). */
int64_t oracle_sgmm(uint64_t n, const int64_t *offsets, const uint32_t *nbrs,
                    uint32_t *mate, uint32_t *pairs)
{
    unsigned char *marked = (unsigned char *)calloc(n ? n : 1, 1);
    if (!marked) return -1;
    for (uint64_t v = 0; v < n; ++v) mate[v] = ORACLE_NONE;

    int64_t taken = 0;
    for (uint64_t x = 0; x < n; ++x) {
        if (marked[x]) continue;                 /* row of a marked source: nothing to take */
        for (int64_t i = offsets[x]; i < offsets[x + 1]; ++i) {
            uint64_t y = nbrs[i];
            if (y >= n) { free(marked); return -1; }
            if (y == x) continue;                /* self-loop */
            if (!marked[y]) {
                marked[x] = 1;
                marked[y] = 1;
                mate[x] = (uint32_t)y;
                mate[y] = (uint32_t)x;
                if (pairs) {
                    pairs[2 * taken]     = (uint32_t)(x < y ? x : y);
                    pairs[2 * taken + 1] = (uint32_t)(x < y ? y : x);
                }
                ++taken;
                break;                           /* x is marked: leave the row */
            }
        }
    }
    free(marked);
    return taken;
}

/* Same computation, timed with a monotonic clock around the edge walk only
 * (the paper times after the graph is loaded, Section VI-B).  *seconds gets
 * the wall time of the walk. */
int64_t oracle_sgmm_timed(uint64_t n, const int64_t *offsets, const uint32_t *nbrs,
                          uint32_t *mate, double *seconds)
{
    struct timespec t0, t1;
    clock_gettime(CLOCK_MONOTONIC, &t0);
    int64_t r = oracle_sgmm(n, offsets, nbrs, mate, NULL);
    clock_gettime(CLOCK_MONOTONIC, &t1);
    *seconds = (double)(t1.tv_sec - t0.tv_sec) + 1e-9 * (double)(t1.tv_nsec - t0.tv_nsec);
    return r;
}

/* SGMM restricted to the rows [row_begin, row_end) of the same graph, with
 * the marks of the earlier rows taken as they stand in `mate` on entry.  Used
 * only to time a bounded sample of a large graph on the host: the caller
 * initialises mate to NONE and calls it once with row_begin = 0. */
int64_t oracle_sgmm_rows_timed(uint64_t n, const int64_t *offsets, const uint32_t *nbrs,
                               uint64_t row_begin, uint64_t row_end,
                               uint32_t *mate, double *seconds)
{
    struct timespec t0, t1;
    clock_gettime(CLOCK_MONOTONIC, &t0);
    int64_t taken = 0;
    for (uint64_t x = row_begin; x < row_end && x < n; ++x) {
        if (mate[x] != ORACLE_NONE) continue;
        for (int64_t i = offsets[x]; i < offsets[x + 1]; ++i) {
            uint64_t y = nbrs[i];
            if (y >= n) return -1;
            if (y == x) continue;
            if (mate[y] == ORACLE_NONE) {
                mate[x] = (uint32_t)y;
                mate[y] = (uint32_t)x;
                ++taken;
                break;
            }
        }
    }
    clock_gettime(CLOCK_MONOTONIC, &t1);
    *seconds = (double)(t1.tv_sec - t0.tv_sec) + 1e-9 * (double)(t1.tv_nsec - t0.tv_nsec);
    return taken;
}
