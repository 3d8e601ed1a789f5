"""Pins for the edge-list oracle (CPU only): oracle.sgmm_edges / check_edges.

Section V-C lets Skipper read its input as a list of edges in coordinate form.
The oracle for that input is SGMM over the list in list order plus the exact
checker with the listed edges as the edge set.  They are pinned here against
things other than themselves:
  * the CSR oracle (itself pinned in test_oracle.py): over the entries of a
    CSR in row order, greedy over the list equals SGMM with its row skip;
  * the worked example of Fig. 1 in list form, in several orders;
  * closed forms (a path listed forwards and backwards, a star in any order,
    K_{a,b} in any order);
  * brute force over every graph on up to five vertices in a random order,
    and over every matching of those graphs for the checker;
  * the CSR checker on the same edge set, field by field.
"""
import random

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests import brute

NONE = oracle.NONE


def _rows_as_list(g):
    off, nb = g.offsets.numpy(), g.nbrs.numpy().view(np.uint32)
    src = np.repeat(np.arange(g.n, dtype=np.uint32), np.diff(off))
    return src, nb


@pytest.mark.parametrize("make", [
    lambda: gg.rmat(9, 8, seed=5),
    lambda: gg.uniform(700, 3000, seed=6),
    lambda: gg.grid(13, 17),
    lambda: gg.star(40),
    lambda: gg.complete(9),
])
def test_list_in_row_order_equals_csr_sgmm(make):
    g = make()
    src, dst = _rows_as_list(g)
    m_csr, p_csr = oracle.sgmm(g.offsets.numpy(), g.nbrs.numpy())
    m_list, p_list = oracle.sgmm_edges(g.n, src, dst)
    assert np.array_equal(m_list, m_csr)
    assert np.array_equal(p_list, p_csr)


def test_worked_example_fig1_as_a_list():
    # Fig. 1's graph, its edges listed in the order SGMM meets them in CSR
    src = [0, 0, 0, 1, 2]
    dst = [1, 2, 3, 2, 3]
    m, p = oracle.sgmm_edges(4, src, dst)
    assert m.tolist() == [1, 0, 3, 2] and p.tolist() == [[0, 1], [2, 3]]
    # reversed list and reversed directions: (2,3) first, then (0,1)
    m, p = oracle.sgmm_edges(4, dst[::-1], src[::-1])
    assert m.tolist() == [1, 0, 3, 2] and p.tolist() == [[2, 3], [0, 1]]
    # (1,2) first leaves (0,3) as the only edge with two free ends
    m, p = oracle.sgmm_edges(4, [1, 0, 0, 0, 2], [2, 1, 2, 3, 3])
    assert m.tolist() == [3, 2, 1, 0] and p.tolist() == [[1, 2], [0, 3]]
    assert oracle.check_edges(4, [1, 0, 0, 0, 2], [2, 1, 2, 3, 3], m, p).flags == 0


@pytest.mark.parametrize("n", [2, 3, 8, 11, 100])
def test_path_forwards_and_backwards(n):
    a = np.arange(n - 1, dtype=np.uint32)
    m, p = oracle.sgmm_edges(n, a, a + 1)
    assert p.tolist() == [[2 * i, 2 * i + 1] for i in range(n // 2)]
    # listed from the far end: (n-2, n-1), (n-4, n-3), ...
    m, p = oracle.sgmm_edges(n, (a + 1)[::-1], a[::-1])
    assert p.tolist() == [[n - 2 - 2 * i, n - 1 - 2 * i] for i in range(n // 2)]
    assert (m[0] == NONE) == (n % 2 == 1)
    assert oracle.check_edges(n, a, a + 1, m, p).flags == 0


@pytest.mark.parametrize("k", [1, 2, 9, 50])
def test_star_any_order_takes_the_first_edge(k):
    rng = random.Random(k)
    leaves = list(range(1, k + 1))
    rng.shuffle(leaves)
    flip = [rng.random() < 0.5 for _ in leaves]
    src = [l if f else 0 for l, f in zip(leaves, flip)]
    dst = [0 if f else l for l, f in zip(leaves, flip)]
    m, p = oracle.sgmm_edges(k + 1, src, dst)
    assert p.tolist() == [[0, leaves[0]]]
    assert oracle.check_edges(k + 1, src, dst, m, p).flags == 0


@pytest.mark.parametrize("a,b", [(1, 1), (2, 5), (6, 3), (7, 7)])
def test_complete_bipartite_any_order(a, b):
    edges = [(i, a + j) for i in range(a) for j in range(b)]
    for seed in range(5):
        random.Random(seed).shuffle(edges)
        src = [e[seed % 2] for e in edges]
        dst = [e[1 - seed % 2] for e in edges]
        m, p = oracle.sgmm_edges(a + b, src, dst)
        assert len(p) == min(a, b)   # every maximal matching of K_{a,b} has min(a, b) edges
        assert oracle.check_edges(a + b, src, dst, m, p).flags == 0


def test_loops_and_repeats():
    src = [0, 1, 1, 2, 0, 3]
    dst = [0, 1, 2, 1, 1, 3]   # loops (0,0) (1,1) (3,3); (1,2) listed twice
    m, p = oracle.sgmm_edges(4, src, dst)
    assert p.tolist() == [[1, 2]] and m[0] == NONE and m[3] == NONE
    v = oracle.check_edges(4, src, dst, m, p)
    assert v.flags == 0 and v.n_uncovered == 0


def test_out_of_range_id_is_refused():
    with pytest.raises(ValueError):
        oracle.sgmm_edges(3, [0, 1], [1, 3])


def _brute_graphs(max_n):
    for n in range(1, max_n + 1):
        for adj in brute.graphs_on(n):
            yield n, adj


def test_brute_force_greedy_is_maximal_in_any_order():
    rng = random.Random(17)
    for n, adj in _brute_graphs(5):
        edges = sorted({tuple(sorted((x, y))) for x in range(n) for y in adj[x]})
        rng.shuffle(edges)
        flip = [rng.random() < 0.5 for _ in edges]
        src = [e[1] if f else e[0] for e, f in zip(edges, flip)]
        dst = [e[0] if f else e[1] for e, f in zip(edges, flip)]
        m, p = oracle.sgmm_edges(n, np.array(src, np.uint32), np.array(dst, np.uint32))
        off, nb = brute.csr_from_adj(n, adj)
        assert brute.mate_is_valid_maximal(n, off, nb, m.tolist())
        es = {frozenset(e) for e in edges}
        assert len(p) * 2 >= brute.maximum_matching_size(es) if es else len(p) == 0


def test_brute_force_checker_accepts_exactly_the_maximal_matchings():
    rng = random.Random(23)
    for n, adj in _brute_graphs(5):
        edges = sorted({tuple(sorted((x, y))) for x in range(n) for y in adj[x]})
        rng.shuffle(edges)
        src = np.array([e[0] for e in edges], np.uint32)
        dst = np.array([e[1] for e in edges], np.uint32)
        es = {frozenset(e) for e in edges}
        for mt in brute.all_matchings(es):
            mate = np.array(brute.mate_of(n, mt), dtype=np.uint32)
            v = oracle.check_edges(n, src, dst, mate)
            assert (v.flags == 0) == brute.is_maximal(es, mt)
            assert v.n_pairs == len(mt) and v.n_matched == 2 * len(mt)


def _csr_once(n, src, dst):
    """CSR holding each listed edge once, in the row of its src (Section V-C)."""
    order = np.lexsort((dst, src))
    s, d = src[order], dst[order]
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, s.astype(np.int64) + 1, 1)
    return np.cumsum(off), d


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_checker_agrees_with_the_csr_checker(seed):
    g = gg.rmat(9, 6, seed=seed)
    src, dst = (t.numpy().view(np.uint32) for t in gg.edge_list(g, "shuffle", seed=seed))
    n = g.n
    good, _ = oracle.sgmm_edges(n, src, dst)
    rng = np.random.default_rng(seed)
    bad_cases = []
    m = good.copy(); v = int(np.flatnonzero(m != NONE)[0]); w = int(m[v]); m[v] = m[w] = NONE
    bad_cases.append(m)
    m = good.copy(); v = int(np.flatnonzero(m != NONE)[1]); m[v] = (m[v] + 1) % n; bad_cases.append(m)
    m = good.copy(); m[int(rng.integers(n))] = n + 5; bad_cases.append(m)
    m = good.copy(); u = int(np.flatnonzero(m == NONE)[0]) if np.any(m == NONE) else 0
    m[u] = u; bad_cases.append(m)
    off, nb = _csr_once(n, src, dst)
    for mate in [good] + bad_cases:
        ve = oracle.check_edges(n, src, dst, mate).as_dict()
        vc = oracle.check(off, nb, mate).as_dict()
        fu = ve.pop("first_uncovered")
        vc.pop("first_uncovered")
        assert ve == vc
        if ve["n_uncovered"]:
            i = fu
            assert mate[src[i]] == NONE and mate[dst[i]] == NONE and src[i] != dst[i]
            early = (mate[src[:i]] == NONE) & (mate[dst[:i]] == NONE) & (src[:i] != dst[:i])
            assert not early.any()


def test_corruptions_each_flag():
    n = 6
    src = np.array([0, 1, 2, 3, 4, 0], np.uint32)
    dst = np.array([1, 2, 3, 4, 5, 5], np.uint32)
    mate, pairs = oracle.sgmm_edges(n, src, dst)     # (0,1) (2,3) (4,5)
    assert pairs.tolist() == [[0, 1], [2, 3], [4, 5]]
    assert oracle.check_edges(n, src, dst, mate, pairs).flags == 0
    m = mate.copy(); m[2] = m[3] = NONE
    v = oracle.check_edges(n, src, dst, m)
    assert v.flags == oracle.V_UNCOVERED and v.n_uncovered == 1 and v.first_uncovered == 2
    m = mate.copy(); m[0] = 2
    assert oracle.check_edges(n, src, dst, m).flags & oracle.V_ASYM
    m = mate.copy(); m[1], m[2] = 2, 1; m[0] = m[3] = NONE
    v = oracle.check_edges(n, src, dst, m)
    assert v.flags == 0     # (1,2) is a listed edge; (0,5) and (3,4) cover the rest
    m = mate.copy(); m[0], m[2] = 2, 0; m[1] = m[3] = NONE
    assert oracle.check_edges(n, src, dst, m).flags & oracle.V_NONEDGE
    m = mate.copy(); m[4] = 9
    v = oracle.check_edges(n, src, dst, m)
    assert v.flags & oracle.V_RANGE and v.first_bad_vertex == 4
    v = oracle.check_edges(n, src, dst, mate, np.array([[0, 1], [0, 1], [2, 3]], np.uint32))
    assert v.flags == oracle.V_PAIRS and v.n_pairs_bad == 1
