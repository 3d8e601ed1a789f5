"""Brute-force maximal-matching facts for tiny graphs (pure Python).

These restate the definitions of Section II-B directly on edge sets, with no
shortcut, so that they can pin the C oracle: a matching is a set of edges no
two of which share an endpoint; it is maximal when every graph edge shares an
endpoint with one of its edges; SGMM as defined in the text walks the edges in
order and takes an edge when neither endpoint is marked.
"""
from itertools import combinations

NONE = 0xFFFFFFFF


def csr_from_adj(n, adj):
    """adj: list of lists (stored order kept)."""
    offsets = [0]
    nbrs = []
    for x in range(n):
        nbrs.extend(adj[x])
        offsets.append(len(nbrs))
    return offsets, nbrs


def undirected_edges(offsets, nbrs):
    n = len(offsets) - 1
    return {frozenset((x, nbrs[i])) for x in range(n) for i in range(offsets[x], offsets[x + 1])
            if nbrs[i] != x}


def all_matchings(edges):
    """Every matching (as a list of frozensets) of the undirected edge set."""
    edges = sorted(edges, key=lambda e: tuple(sorted(e)))
    out = []

    def rec(i, used, cur):
        if i == len(edges):
            out.append(list(cur))
            return
        rec(i + 1, used, cur)
        e = edges[i]
        if not (e & used):
            cur.append(e)
            rec(i + 1, used | e, cur)
            cur.pop()

    rec(0, frozenset(), [])
    return out


def is_maximal(edges, matching):
    covered = set()
    for e in matching:
        covered |= e
    return all(e & covered for e in edges)


def maximum_matching_size(edges):
    return max(len(m) for m in all_matchings(edges))


def mate_of(n, matching):
    mate = [NONE] * n
    for e in matching:
        a, b = sorted(e)
        mate[a], mate[b] = b, a
    return mate


def mate_is_valid_maximal(n, offsets, nbrs, mate):
    """Section II-B's rule on the edge set a mate array names."""
    edges = undirected_edges(offsets, nbrs)
    out = set()
    for v in range(n):
        m = mate[v]
        if m == NONE:
            continue
        if m >= n or m == v:
            return False
        out.add(frozenset((v, m)))
    # every output edge must exist in the graph
    if not out <= edges:
        return False
    # (b) no two output edges share an endpoint; and every vertex in an
    # output edge must name that edge's other endpoint
    seen = {}
    for e in out:
        for v in e:
            if v in seen:
                return False
            seen[v] = e
    for v in range(n):
        if v in seen:
            (w,) = seen[v] - {v}
            if mate[v] != w:
                return False
        elif mate[v] != NONE:
            return False
    # (a) every graph edge touches an output edge
    return is_maximal(edges, out)


def greedy_edge_walk(n, offsets, nbrs):
    """SGMM exactly as worded: walk every stored edge, take it if both ends unmarked."""
    marked = [False] * n
    mate = [NONE] * n
    pairs = []
    for x in range(n):
        for i in range(offsets[x], offsets[x + 1]):
            y = nbrs[i]
            if y == x:
                continue
            if not marked[x] and not marked[y]:
                marked[x] = marked[y] = True
                mate[x], mate[y] = y, x
                pairs.append((min(x, y), max(x, y)))
    return mate, pairs


def graphs_on(n):
    """Every simple undirected graph on n labelled vertices, as sorted adjacency lists."""
    slots = list(combinations(range(n), 2))
    for mask in range(1 << len(slots)):
        adj = [[] for _ in range(n)]
        for k, (a, b) in enumerate(slots):
            if mask >> k & 1:
                adj[a].append(b)
                adj[b].append(a)
        for row in adj:
            row.sort()
        yield adj
