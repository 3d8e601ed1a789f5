"""Pins for the oracle (CPU only): the worked example, closed forms, brute force.

The oracle (oracle/) is the reference for every GPU parity test, so it is
pinned here against things other than itself:
  * the worked example the paper walks through (Section II-B, Fig. 1),
  * closed forms of SGMM on graphs with known structure,
  * brute force over every graph on up to six vertices (the definitions of
    Section II-B restated on edge sets in tests/brute.py),
  * SGMM exactly as worded (walk every edge, no row skip).
"""
import os
import random

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests import brute

NONE = oracle.NONE
HERE = os.path.dirname(os.path.abspath(__file__))


def _csr_np(g):
    return g.offsets.numpy(), g.nbrs.numpy()


def _load_golden(name):
    n, edges, mate, pairs = None, [], None, []
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            if line[0] == "n":
                n = int(line[1])
            elif line[0] == "edge":
                edges.append((int(line[1]), int(line[2])))
            elif line[0] == "mate":
                mate = [int(t) for t in line[1:]]
            elif line[0] == "pair":
                pairs.append((int(line[1]), int(line[2])))
    return n, edges, mate, pairs


def test_worked_example_fig1():
    n, edges, mate, pairs = _load_golden("fig1_worked_example.txt")
    g = gg.from_edges(n, np.array([e[0] for e in edges]), np.array([e[1] for e in edges]))
    off, nb = _csr_np(g)
    m, p = oracle.sgmm(off, nb)
    assert m.tolist() == mate
    assert [tuple(r) for r in p.tolist()] == pairs
    v = oracle.check(off, nb, m, p)
    assert v.flags == 0 and v.n_pairs == 2 and v.n_matched == 4


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 7, 10, 101])
def test_path_closed_form(n):
    off, nb = _csr_np(gg.path(n))
    m, p = oracle.sgmm(off, nb)
    assert [tuple(r) for r in p.tolist()] == [(2 * i, 2 * i + 1) for i in range(n // 2)]
    expect = [(v ^ 1) if (v ^ 1) < n else NONE for v in range(n)]
    assert m.tolist() == expect
    assert oracle.check(off, nb, m, p).flags == 0


@pytest.mark.parametrize("k", [1, 2, 5, 64])
def test_star_closed_form(k):
    off, nb = _csr_np(gg.star(k))
    m, p = oracle.sgmm(off, nb)
    assert p.tolist() == [[0, 1]]
    assert oracle.check(off, nb, m, p).flags == 0


@pytest.mark.parametrize("a,b", [(1, 1), (2, 3), (5, 2), (8, 8), (3, 17)])
def test_complete_bipartite_closed_form(a, b):
    off, nb = _csr_np(gg.complete_bipartite(a, b))
    m, p = oracle.sgmm(off, nb)
    # left vertex i meets the right vertices a..a+b-1 in order; a+i is the first free one
    assert [tuple(r) for r in p.tolist()] == [(i, a + i) for i in range(min(a, b))]
    assert oracle.check(off, nb, m, p).flags == 0


@pytest.mark.parametrize("k", [1, 3, 50])
def test_disjoint_edges_closed_form(k):
    off, nb = _csr_np(gg.disjoint_edges(k))
    m, p = oracle.sgmm(off, nb)
    assert m.tolist() == [v ^ 1 for v in range(2 * k)]
    assert oracle.check(off, nb, m, p).flags == 0


@pytest.mark.parametrize("n", [2, 3, 6, 9])
def test_complete_graph_closed_form(n):
    off, nb = _csr_np(gg.complete(n))
    m, p = oracle.sgmm(off, nb)
    assert [tuple(r) for r in p.tolist()] == [(2 * i, 2 * i + 1) for i in range(n // 2)]


@pytest.mark.parametrize("rows,cols", [(1, 2), (2, 2), (3, 4), (16, 32), (5, 6)])
def test_grid_closed_form(rows, cols):
    off, nb = _csr_np(gg.grid(rows, cols))
    m, p = oracle.sgmm(off, nb)
    expect = [(r * cols + 2 * c, r * cols + 2 * c + 1) for r in range(rows) for c in range(cols // 2)]
    assert [tuple(x) for x in p.tolist()] == expect
    assert len(expect) * 2 == rows * cols  # perfect on even widths


def test_self_loops_and_stored_order():
    # row 0 lists a self-loop first and then 2 before 1: SGMM skips the loop and
    # takes the first free neighbour in stored order.
    off = [0, 3, 4, 5]
    nb = [0, 2, 1, 0, 0]
    m, p = oracle.sgmm(off, nb)
    assert m.tolist() == [2, NONE, 0]
    assert p.tolist() == [[0, 2]]


def test_checker_ignores_self_loops():
    """A loop is not an edge a matching can cover (Algorithm 1 lines 6-7 skip
    it): an unmatched vertex whose only entry is a loop leaves nothing
    uncovered, while a real edge between two unmatched vertices is reported."""
    # 0 - 1 matched; vertex 2 has only a loop; vertex 3 a loop and the edge 3-4
    off = [0, 1, 2, 3, 5, 6]
    nb = [1, 0, 2, 3, 4, 3]
    mate = np.array([1, 0, NONE, 4, 3], dtype=np.uint32)
    v = oracle.check(off, nb, mate)
    assert v.flags == 0 and v.n_uncovered == 0 and v.n_pairs == 2
    mate = np.array([1, 0, NONE, NONE, NONE], dtype=np.uint32)
    v = oracle.check(off, nb, mate)
    assert v.flags == oracle.V_UNCOVERED and v.n_uncovered == 2   # entries 3->4 and 4->3
    m, _ = oracle.sgmm(off, nb)
    assert m.tolist() == [1, 0, NONE, 4, 3]
    assert oracle.check(off, nb, m).flags == 0


def test_sgmm_equals_edge_walk_random():
    rng = random.Random(7)
    for _ in range(300):
        n = rng.randint(1, 12)
        adj = [[] for _ in range(n)]
        for x in range(n):
            for _ in range(rng.randint(0, 5)):
                adj[x].append(rng.randrange(n))   # loops, repeats, any order
        off, nb = brute.csr_from_adj(n, adj)
        m, p = oracle.sgmm(off, nb)
        bm, bp = brute.greedy_edge_walk(n, off, nb)
        assert m.tolist() == bm
        assert [tuple(r) for r in p.tolist()] == bp


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_sgmm_equals_edge_walk_generated(seed):
    g = gg.rmat(9, 8, seed=seed)
    off, nb = _csr_np(g)
    m, p = oracle.sgmm(off, nb)
    bm, bp = brute.greedy_edge_walk(g.n, off.tolist(), nb.tolist())
    assert m.tolist() == bm
    # on a symmetric CSR SGMM takes its matches in ascending order of the lower end
    assert [tuple(r) for r in p.tolist()] == bp
    assert all(p[i, 0] < p[i + 1, 0] for i in range(len(p) - 1))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_exhaustive_small_graphs(n):
    for adj in brute.graphs_on(n):
        off, nb = brute.csr_from_adj(n, adj)
        edges = brute.undirected_edges(off, nb)
        m, p = oracle.sgmm(off, nb)
        out = [frozenset((int(a), int(b))) for a, b in p.tolist()]
        assert brute.is_maximal(edges, out)
        assert brute.mate_is_valid_maximal(n, off, nb, m.tolist())
        nu = brute.maximum_matching_size(edges)
        assert 2 * len(out) >= nu
        assert oracle.check(off, nb, m, p).flags == 0


def test_exhaustive_six_vertices():
    n = 6
    for adj in brute.graphs_on(n):
        off, nb = brute.csr_from_adj(n, adj)
        edges = brute.undirected_edges(off, nb)
        m, _ = oracle.sgmm(off, nb)
        out = [frozenset((v, int(m[v]))) for v in range(n) if m[v] != NONE and v < m[v]]
        assert brute.is_maximal(edges, out)
        assert oracle.check(off, nb, m).flags == 0


def test_sampled_seven_vertices():
    """Seeded random graphs on 7 vertices (random edge subsets of the 21 pairs,
    rows in random stored order): SGMM's result is maximal and at least half a
    maximum matching; every matching of the graph is accepted by the checker
    exactly when it is maximal."""
    rng = random.Random(17)
    n = 7
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    for t in range(1500):
        adj = [[] for _ in range(n)]
        for a, b in pairs:
            if rng.random() < rng.choice((0.2, 0.45, 0.7)):
                adj[a].append(b)
                adj[b].append(a)
        for row in adj:
            rng.shuffle(row)
        off, nb = brute.csr_from_adj(n, adj)
        edges = brute.undirected_edges(off, nb)
        m, p = oracle.sgmm(off, nb)
        out = [frozenset((int(a), int(b))) for a, b in p.tolist()]
        assert brute.is_maximal(edges, out)
        assert 2 * len(out) >= brute.maximum_matching_size(edges)
        assert oracle.check(off, nb, m, p).flags == 0
        if t % 10 == 0:
            for mt in brute.all_matchings(edges):
                v = oracle.check(off, nb, np.array(brute.mate_of(n, mt), dtype=np.uint32))
                assert (v.flags == 0) == brute.is_maximal(edges, mt)


@pytest.mark.parametrize("n", [3, 4])
def test_checker_accepts_exactly_the_maximal_matchings(n):
    """Every mate array over {NONE, 0..n-1} on every graph: accepted iff Section II-B holds."""
    import itertools
    vals = [NONE] + list(range(n))
    for adj in brute.graphs_on(n):
        off, nb = brute.csr_from_adj(n, adj)
        for mate in itertools.product(vals, repeat=n):
            ok = brute.mate_is_valid_maximal(n, off, nb, list(mate))
            v = oracle.check(off, nb, np.array(mate, dtype=np.uint32))
            assert (v.flags == 0) == ok, (adj, mate, v.as_dict())


@pytest.mark.parametrize("n", [3, 4])
def test_checker_on_edges_stored_once(n):
    """Each edge kept only in the row of its lower end (Section V-C): the checker
    still accepts exactly the maximal matchings of the edge set."""
    import itertools
    vals = [NONE] + list(range(n))
    for adj in brute.graphs_on(n):
        once = [[y for y in adj[x] if y > x] for x in range(n)]
        off, nb = brute.csr_from_adj(n, once)
        for mate in itertools.product(vals, repeat=n):
            ok = brute.mate_is_valid_maximal(n, off, nb, list(mate))
            v = oracle.check(off, nb, np.array(mate, dtype=np.uint32))
            assert (v.flags == 0) == ok, (once, mate, v.as_dict())
        m, p = oracle.sgmm(off, nb)
        assert brute.mate_is_valid_maximal(n, off, nb, m.tolist())


def test_every_maximal_matching_within_half_of_maximum():
    rng = random.Random(3)
    for _ in range(60):
        n = rng.randint(2, 7)
        adj = [[] for _ in range(n)]
        for a in range(n):
            for b in range(a + 1, n):
                if rng.random() < 0.45:
                    adj[a].append(b)
                    adj[b].append(a)
        off, nb = brute.csr_from_adj(n, adj)
        edges = brute.undirected_edges(off, nb)
        nu = brute.maximum_matching_size(edges)
        for mt in brute.all_matchings(edges):
            v = oracle.check(off, nb, np.array(brute.mate_of(n, mt), dtype=np.uint32))
            if brute.is_maximal(edges, mt):
                assert v.flags == 0 and nu <= 2 * len(mt) <= 2 * nu
            else:
                assert v.flags == oracle.V_UNCOVERED


def test_checker_counts_on_corruptions():
    g = gg.path(6)          # 0-1-2-3-4-5
    off, nb = _csr_np(g)
    good = np.array([1, 0, 3, 2, 5, 4], dtype=np.uint32)
    assert oracle.check(off, nb, good).flags == 0

    drop = good.copy(); drop[2] = drop[3] = NONE          # edge (2,3) uncovered
    v = oracle.check(off, nb, drop)
    assert v.flags == oracle.V_UNCOVERED and v.n_uncovered == 2
    assert v.first_uncovered == off[2] + 1                 # entry (2,3) in row 2

    asym = good.copy(); asym[4] = NONE                      # 5 names 4, 4 names nobody
    v = oracle.check(off, nb, asym)
    assert v.flags == oracle.V_ASYM and v.n_asym == 1 and v.first_bad_vertex == 5

    rng_ = good.copy(); rng_[1] = 99                        # 1 names a vertex outside [0, n)
    v = oracle.check(off, nb, rng_)                          # ... and 0 is left asymmetric
    assert v.flags == oracle.V_RANGE | oracle.V_ASYM
    assert (v.n_bad_range, v.n_asym, v.first_bad_vertex) == (1, 1, 0)

    self_ = good.copy(); self_[0] = 0                       # 0 names itself
    v = oracle.check(off, nb, self_)
    assert v.flags == oracle.V_RANGE | oracle.V_ASYM
    assert (v.n_bad_range, v.n_asym, v.first_bad_vertex) == (1, 1, 0)

    nonedge = np.array([2, NONE, 0, 4, 3, NONE], dtype=np.uint32)   # (0,2) is not an edge
    v = oracle.check(off, nb, nonedge)
    assert v.flags == oracle.V_NONEDGE and v.n_nonedge == 2 and v.first_bad_vertex == 0

    dup = np.array([1, 0, 1, NONE, 5, 4], dtype=np.uint32)  # 1 claimed by 0 and 2
    v = oracle.check(off, nb, dup)
    assert v.flags & oracle.V_ASYM and v.n_asym == 1 and v.first_bad_vertex == 2


def test_checker_pairs_list():
    off, nb = _csr_np(gg.path(6))
    mate = np.array([1, 0, 3, 2, 5, 4], dtype=np.uint32)
    good = np.array([[0, 1], [2, 3], [4, 5]], dtype=np.uint32)
    assert oracle.check(off, nb, mate, good).flags == 0
    assert oracle.check(off, nb, mate, good[[2, 0, 1]]).flags == 0       # any order
    v = oracle.check(off, nb, mate, good[:2])                              # one missing
    assert v.flags == oracle.V_PAIRS and v.n_pairs_bad == 0
    v = oracle.check(off, nb, mate, np.array([[0, 1], [0, 1], [2, 3]], dtype=np.uint32))
    assert v.flags == oracle.V_PAIRS and v.n_pairs_bad == 1               # repeat
    v = oracle.check(off, nb, mate, np.array([[1, 0], [2, 3], [4, 5]], dtype=np.uint32))
    assert v.flags == oracle.V_PAIRS and v.n_pairs_bad == 1               # not (low, high)
    v = oracle.check(off, nb, mate, np.zeros((0, 2), dtype=np.uint32))
    assert v.flags == oracle.V_PAIRS


def test_sgmm_on_er_generated():
    g = gg.erdos_renyi(2000, 9000, seed=11)
    off, nb = _csr_np(g)
    m, p = oracle.sgmm(off, nb)
    v = oracle.check(off, nb, m, p)
    assert v.flags == 0 and v.n_pairs == len(p) and v.n_matched == 2 * len(p)
