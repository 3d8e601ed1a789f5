/*
 * oracle/check.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Exact checker for a maximal-matching result, written from the paper's
 * validation rule in Section II-B: (a) every graph edge shares an endpoint
 * with an output edge, and (b) no two output edges share an endpoint.  The
 * output is given as a per-vertex mate array (0xFFFFFFFF = unmatched) and,
 * optionally, as a list of (u, v) pairs.
 *
 * With a mate array, (b) is the symmetry rule mate[mate[v]] == v: a vertex
 * can name only one partner, so a symmetric mate array is a set of disjoint
 * pairs.  Each named partner must also be a neighbour: the output edge must
 * exist in the graph, stored in the row of either endpoint (Section V-C lets
 * a CSR hold an edge for one endpoint only).  (a) is checked over every stored
 * CSR entry.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * call this file.  It shares no code with the CUDA library.
 *
 * Counting rules (the CUDA validator has to reproduce them exactly):
 *   for every v with m = mate[v] != NONE:
 *     m >= n or m == v           -> n_bad_range, v is a bad vertex
 *     else n_matched += 1, and
 *       mate[m] != v             -> n_asym,      v is a bad vertex
 *       m not in row v and v not in row m -> n_nonedge, v is a bad vertex
 *   n_pairs = #{v : m = mate[v] in range, v < m, mate[m] == v}
 *   for every entry i of row x with y = nbrs[i], y != x:
 *     mate[x] == NONE and mate[y] == NONE -> n_uncovered (first = min i)
 *   pairs list (when given): a pair (a, b) is valid when a < b < n,
 *     mate[a] == b and mate[b] == a; n_pairs_bad counts the invalid pairs
 *     plus the repeats of a valid pair; the PAIRS flag is set when
 *     n_pairs_bad > 0 or the count differs from n_pairs.
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
} oracle_verdict;

static int row_contains(const int64_t *offsets, const uint32_t *nbrs, uint64_t v, uint64_t w)
{
    for (int64_t i = offsets[v]; i < offsets[v + 1]; ++i)
        if ((uint64_t)nbrs[i] == w) return 1;
    return 0;
}

/* Returns 0, or -1 when memory for the pair marks cannot be had. */
int oracle_check(uint64_t n, const int64_t *offsets, const uint32_t *nbrs,
                 const uint32_t *mate, const uint32_t *pairs, uint64_t count,
                 oracle_verdict *out)
{
    oracle_verdict r;
    memset(&r, 0, sizeof r);
    r.first_bad_vertex = UINT64_MAX;
    r.first_uncovered = UINT64_MAX;

    for (uint64_t v = 0; v < n; ++v) {
        uint64_t m = mate[v];
        if (m == ORACLE_NONE) continue;
        int bad = 0;
        if (m >= n || m == v) {
            r.n_bad_range++;
            bad = 1;
        } else {
            r.n_matched++;
            if ((uint64_t)mate[m] != v) { r.n_asym++; bad = 1; }
            else if (v < m) r.n_pairs++;
            if (!row_contains(offsets, nbrs, v, m) && !row_contains(offsets, nbrs, m, v)) {
                r.n_nonedge++;
                bad = 1;
            }
        }
        if (bad && v < r.first_bad_vertex) r.first_bad_vertex = v;
    }

    for (uint64_t x = 0; x < n; ++x) {
        if (mate[x] != ORACLE_NONE) continue;
        for (int64_t i = offsets[x]; i < offsets[x + 1]; ++i) {
            uint64_t y = nbrs[i];
            if (y == x) continue;
            if (mate[y] == ORACLE_NONE) {
                r.n_uncovered++;
                if ((uint64_t)i < r.first_uncovered) r.first_uncovered = (uint64_t)i;
            }
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
