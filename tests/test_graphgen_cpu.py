"""The seeded generators (CPU): the CSR build gives the same graph for any
number of source-range chunks (large graphs are built in chunks to bound
their temporaries), and a graph is a symmetric CSR with sorted, de-duplicated
rows and no loops."""
import numpy as np
import pytest

import graphgen as gg


def _same(a, b):
    assert a.n == b.n and a.nnz == b.nnz
    assert np.array_equal(a.offsets.numpy(), b.offsets.numpy())
    assert np.array_equal(a.nbrs.numpy(), b.nbrs.numpy())


@pytest.mark.parametrize("chunks", [2, 5, 16, 64])
def test_chunked_build_is_the_same_graph(chunks):
    _same(gg.rmat(12, 8, seed=3), gg.rmat(12, 8, seed=3, chunks=chunks))
    _same(gg.uniform(3000, 20000, seed=4), gg.uniform(3000, 20000, seed=4, chunks=chunks))
    _same(gg.rmat(10, 16, .7, .1, .1, seed=5), gg.rmat(10, 16, .7, .1, .1, seed=5, chunks=chunks))


def test_csr_shape():
    for g in (gg.rmat(11, 16, seed=1), gg.uniform(2000, 9000, seed=2)):
        off, nb = g.offsets.numpy(), g.nbrs.numpy().astype(np.int64)
        assert off[0] == 0 and off[-1] == g.nnz and np.all(np.diff(off) >= 0)
        rows = np.repeat(np.arange(g.n), np.diff(off))
        assert np.all(nb != rows)                                  # no loops
        assert np.all((nb >= 0) & (nb < g.n))
        same_row = rows[1:] == rows[:-1]
        assert np.all(nb[1:][same_row] > nb[:-1][same_row])       # sorted, no repeats
        fwd = set(zip(rows.tolist(), nb.tolist()))
        assert all((y, x) in fwd for x, y in fwd)                  # symmetric


def test_seeds_differ_and_repeat():
    a, b = gg.rmat(10, 8, seed=1), gg.rmat(10, 8, seed=2)
    assert not (a.nnz == b.nnz and np.array_equal(a.nbrs.numpy(), b.nbrs.numpy()))
    _same(a, gg.rmat(10, 8, seed=1))
