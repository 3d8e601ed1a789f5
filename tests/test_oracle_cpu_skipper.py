"""The host-thread Skipper baseline (oracle.cpu_skipper), CPU only.

It is a benchmark baseline, not an oracle, so it is held to the oracle: on
one thread, rows in order, Algorithm 1 takes exactly SGMM's edges in CSR
order (every entry is tested at line 10, so with or without the row skip the
result is SGMM's); on several threads every result must be a maximal matching
by the oracle's checker, with the size fixed where every maximal matching has
one size (star, K_{a,b}, K_n) or the matching is unique (disjoint edges).
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

NONE = oracle.NONE

GRAPHS = {
    "rmat14": lambda: gg.rmat(14, 16, seed=3),
    "uniform": lambda: gg.uniform(20000, 100000, seed=4),
    "grid": lambda: gg.grid(64, 96),
    "path": lambda: gg.path(5001),
    "star": lambda: gg.star(3000),
    "k40_70": lambda: gg.complete_bipartite(40, 70),
    "k33": lambda: gg.complete(33),
    "disjoint": lambda: gg.disjoint_edges(2000),
}


@pytest.mark.parametrize("row_skip", [False, True])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_one_thread_is_sgmm(name, row_skip):
    g = GRAPHS[name]()
    off, nb = g.offsets.numpy(), g.nbrs.numpy()
    ref, _ = oracle.sgmm(off, nb)
    mate, sec, cnf = oracle.cpu_skipper(off, nb, 1, row_skip, block_edges=1000)
    assert np.array_equal(mate, ref) and cnf == 0 and sec >= 0


@pytest.mark.parametrize("threads", [2, 4, 8])
@pytest.mark.parametrize("row_skip", [False, True])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_threads_give_a_maximal_matching(name, row_skip, threads):
    g = GRAPHS[name]()
    off, nb = g.offsets.numpy(), g.nbrs.numpy()
    mate, _, _ = oracle.cpu_skipper(off, nb, threads, row_skip, block_edges=512)
    v = oracle.check(off, nb, mate)
    assert v.flags == 0, v.as_dict()
    _, ref_pairs = oracle.sgmm(off, nb)
    assert 2 * v.n_pairs >= len(ref_pairs)
    fixed = {"star": 1, "k40_70": 40, "k33": 16, "disjoint": 2000}
    if name in fixed:
        assert v.n_pairs == fixed[name]


def test_row_sample_matches_sgmm_over_the_same_rows():
    g = gg.rmat(15, 16, seed=8)
    off, nb = g.offsets.numpy(), g.nbrs.numpy()
    rows = g.n // 3
    k, _, entries = oracle.sgmm_rows_timed(off, nb, rows)
    mate, _, _ = oracle.cpu_skipper(off, nb, 1, False, rows=(0, rows))
    assert int((mate != NONE).sum()) == 2 * k and entries == int(off[rows])
