/*
 * oracle/edges.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Maximal matching over a list of edges in coordinate (COO) form: edge i is
 * (src[i], dst[i]).  Section V-C notes that Skipper needs no particular input
 * format and may read such a list directly; each edge appears once, in either
 * direction.
 *
 * oracle_sgmm_edges: SGMM (Section II-B) over the list in list order -- an
 * edge whose two endpoints are both unmarked is taken and both are marked.
 * Self-loops are never taken (Alg. 1 skips them).  Over the entries of a CSR
 * in row order this is exactly the CSR SGMM of sgmm.c: that one only leaves
 * the rest of a row whose source is marked, and every such entry would be
 * refused here as well.
 *
 * oracle_check_edges: the exact checker of check.c (Section II-B's rule) with
 * the edge list as the edge set.  Counting rules (the CUDA validator has to
 * reproduce them exactly):
 *   for every v with m = mate[v] != NONE:
 *     m >= n or m == v           -> n_bad_range, v is a bad vertex
 *     else n_matched += 1, and
 *       mate[m] != v             -> n_asym,      v is a bad vertex
 *       {v, m} not a list edge   -> n_nonedge,   v is a bad vertex
 *   n_pairs = #{v : m = mate[v] in range, v < m, mate[m] == v}
 *   for every edge i = (x, y), x != y, both ids < n:
 *     mate[x] == NONE and mate[y] == NONE -> n_uncovered (first = min i)
 *   pairs list: as in check.c.
 * Edges with an id >= n are not graph edges and are ignored (the library
 * rejects them before a pass).  Whether {v, m} is a list edge is decided by
 * binary search in the sorted list of (min, max) keys.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * call this file.  It shares no code with the CUDA library.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_NONE 0xFFFFFFFFu

enum {
    ORACLE_V_RANGE     = 1u,
    ORACLE_V_ASYM      = 2u,
    ORACLE_V_NONEDGE   = 4u,
    ORACLE_V_UNCOVERED = 8u,
    ORACLE_V_PAIRS     = 16u,
};

typedef struct {
    uint32_t flags;
    uint32_t pad;
    uint64_t n_matched;
    uint64_t n_pairs;
    uint64_t n_bad_range;
    uint64_t n_asym;
    uint64_t n_nonedge;
    uint64_t n_uncovered;
    uint64_t n_pairs_bad;
    uint64_t first_bad_vertex;
    uint64_t first_uncovered;
} oracle_edges_verdict;

/* Returns the number of matched pairs, or -1 on allocation failure or an
 * endpoint id outside [0, n). */
int64_t oracle_sgmm_edges(uint64_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                          uint32_t *mate, uint32_t *pairs)
{
    unsigned char *marked = (unsigned char *)calloc(n ? n : 1, 1);
    if (!marked) return -1;
    for (uint64_t v = 0; v < n; ++v) mate[v] = ORACLE_NONE;

    int64_t taken = 0;
    for (uint64_t i = 0; i < m; ++i) {
        uint64_t x = src[i], y = dst[i];
        if (x >= n || y >= n) { free(marked); return -1; }
        if (x == y) continue;                       /* self-loop */
        if (marked[x] || marked[y]) continue;
        marked[x] = 1;
        marked[y] = 1;
        mate[x] = (uint32_t)y;
        mate[y] = (uint32_t)x;
        if (pairs) {
            pairs[2 * taken]     = (uint32_t)(x < y ? x : y);
            pairs[2 * taken + 1] = (uint32_t)(x < y ? y : x);
        }
        ++taken;
    }
    free(marked);
    return taken;
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static uint64_t edge_key(uint64_t a, uint64_t b)
{
    return a < b ? (a << 32) | b : (b << 32) | a;
}

/* Returns 0, or -1 when memory cannot be had. */
int oracle_check_edges(uint64_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                       const uint32_t *mate, const uint32_t *pairs, uint64_t count,
                       oracle_edges_verdict *out)
{
    oracle_edges_verdict r;
    memset(&r, 0, sizeof r);
    r.first_bad_vertex = UINT64_MAX;
    r.first_uncovered = UINT64_MAX;

    uint64_t *keys = (uint64_t *)malloc((m ? m : 1) * sizeof(uint64_t));
    if (!keys) return -1;
    uint64_t k = 0;
    for (uint64_t i = 0; i < m; ++i) {
        uint64_t x = src[i], y = dst[i];
        if (x >= n || y >= n || x == y) continue;
        keys[k++] = edge_key(x, y);
    }
    qsort(keys, k, sizeof(uint64_t), cmp_u64);

    for (uint64_t v = 0; v < n; ++v) {
        uint64_t w = mate[v];
        if (w == ORACLE_NONE) continue;
        int bad = 0;
        if (w >= n || w == v) {
            r.n_bad_range++;
            bad = 1;
        } else {
            r.n_matched++;
            if ((uint64_t)mate[w] != v) { r.n_asym++; bad = 1; }
            else if (v < w) r.n_pairs++;
            uint64_t key = edge_key(v, w);
            if (!bsearch(&key, keys, k, sizeof(uint64_t), cmp_u64)) {
                r.n_nonedge++;
                bad = 1;
            }
        }
        if (bad && v < r.first_bad_vertex) r.first_bad_vertex = v;
    }
    free(keys);

    for (uint64_t i = 0; i < m; ++i) {
        uint64_t x = src[i], y = dst[i];
        if (x >= n || y >= n || x == y) continue;
        if (mate[x] == ORACLE_NONE && mate[y] == ORACLE_NONE) {
            r.n_uncovered++;
            if (i < r.first_uncovered) r.first_uncovered = i;
        }
    }

    if (pairs) {
        unsigned char *seen = (unsigned char *)calloc(n ? n : 1, 1);
        if (!seen) return -1;
        for (uint64_t j = 0; j < count; ++j) {
            uint64_t a = pairs[2 * j], b = pairs[2 * j + 1];
            int valid = a < b && b < n && (uint64_t)mate[a] == b && (uint64_t)mate[b] == a;
            if (!valid) { r.n_pairs_bad++; continue; }
            if (seen[a]) r.n_pairs_bad++;
            seen[a] = 1;
        }
        free(seen);
        if (r.n_pairs_bad || count != r.n_pairs) r.flags |= ORACLE_V_PAIRS;
    }

    if (r.n_bad_range) r.flags |= ORACLE_V_RANGE;
    if (r.n_asym) r.flags |= ORACLE_V_ASYM;
    if (r.n_nonedge) r.flags |= ORACLE_V_NONEDGE;
    if (r.n_uncovered) r.flags |= ORACLE_V_UNCOVERED;
    *out = r;
    return 0;
}
