"""Full-size parity at R-MAT scale 27 (ef 16: 134M vertices, ~4.2G CSR entries;
2^31 listed edges for the edge-list input) and at the size of the benchmark's
4096-graph batch, in the launch configurations the benchmark times.

Every result is checked by the oracle's exact checker on the host, over the
whole graph (Section II-B's definition: every edge has a matched endpoint, no
two output edges share an endpoint, every output edge exists), and the device
checker's verdict must equal the oracle's field by field.  Beside it: the
oracle's sequential greedy matching on the same CSR, whose size is at most
twice any maximal matching's (both are maximal), and host-side properties on
sampled vertices (plain numpy, independent of both checkers).
"""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from tests.conftest import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

NONE = 0xFFFFFFFF
SCALE, EF = 27, 16
BENCH_OPTS = dict(status_bits=8, grain=8192, block_threads=512)       # the CSR line of the benchmark
BENCH_COO_OPTS = dict(status_bits=2, grain=8192, block_threads=512)   # its edge-list line


@pytest.fixture(scope="module")
def skp():
    import paper_2507_04420_gb300 as m
    torch.cuda.set_device(0)
    return m


@pytest.fixture(scope="module")
def rmat27():
    g = gg.rmat(SCALE, EF, seed=1, device="cuda", chunks=16)
    yield g
    del g
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def rmat27_host(rmat27):
    """The same CSR in pinned host memory (numpy views for the oracle; the
    tensors serve the in-place path), with the oracle's SGMM pair count."""
    h_off = rmat27.offsets.cpu().pin_memory()
    h_nb = rmat27.nbrs.cpu().pin_memory()
    off, nb = h_off.numpy(), h_nb.numpy()
    _, sgmm_pairs = oracle.sgmm(off, nb)
    yield h_off, h_nb, off, nb, len(sgmm_pairs)
    del h_off, h_nb, off, nb


def _sampled_rows(g, verts):
    """Neighbour lists of the sampled vertices: (row index per entry, ids), on the host."""
    v = torch.from_numpy(verts).cuda()
    starts, ends = g.offsets[v], g.offsets[v + 1]
    lens = ends - starts
    total = int(lens.sum())
    row = torch.repeat_interleave(torch.arange(len(verts), device="cuda"), lens)
    first = torch.cumsum(lens, 0) - lens
    idx = starts[row] + torch.arange(total, device="cuda") - first[row]
    ys = g.nbrs[idx.long()]
    return row.cpu().numpy(), ys.cpu().numpy().view(np.uint32)


def _check_sampled_vertices(g, mate, k, seed):
    n = g.n
    rng = np.random.default_rng(seed)
    verts = rng.choice(n, size=k, replace=False).astype(np.int64)
    row, ys = _sampled_rows(g, verts)
    mv = mate[verts]
    matched = mv != NONE
    # a named partner is in range and names the vertex back
    w = mv[matched].astype(np.int64)
    assert np.all(w < n)
    assert np.all(mate[w] == verts[matched])
    # ... and is a neighbour (the CSR is symmetric: row v holds every edge of v)
    hit = np.zeros(k, dtype=bool)
    np.logical_or.at(hit, row, ys == mv[row])
    assert np.all(hit[matched])
    # an unmatched vertex has every neighbour matched (loops aside)
    free_rows = ~matched[row] & (ys != verts[row])
    assert np.all(mate[ys[free_rows]] != NONE)
    return int(matched.sum())


def _oracle_agrees(off, nb, mate_np, device_verdict, sgmm_pairs):
    vr = oracle.check(off, nb, mate_np)
    assert vr.flags == 0, vr.as_dict()
    assert device_verdict.as_dict() == vr.as_dict(), (device_verdict.as_dict(), vr.as_dict())
    assert 2 * vr.n_pairs >= sgmm_pairs            # |M_SGMM| <= nu <= 2 |M|
    assert 2 * vr.n_pairs == int((mate_np != NONE).sum())
    return vr


@pytest.mark.parametrize("symmetric", [0, 1])
def test_csr_rmat27_in_the_benchmark_launch(skp, rmat27, rmat27_host, symmetric):
    g = rmat27
    _, _, off, nb, sgmm_pairs = rmat27_host
    with skp.Graph(g.offsets, g.nbrs, check=False) as h:
        mate = h.skipper(symmetric=symmetric, **BENCH_OPTS)
        v = h.validate(mate)
    m = mate.cpu().numpy().view(np.uint32)
    _oracle_agrees(off, nb, m, v, sgmm_pairs)
    assert _check_sampled_vertices(g, m, 200_000, seed=3 + symmetric) > 0


def test_csr_rmat27_read_in_place_from_host_memory(skp, rmat27, rmat27_host):
    """The end-to-end path of the benchmark: the CSR in pinned host memory, read
    in place by the kernels (MM_HOST_MAPPED) through the host session, the grain
    chosen by the library; once with the result copied back after the pass (the
    benchmark's line) and once copied back in three pieces while it runs."""
    g = rmat27
    h_off, h_nb, off, nb, sgmm_pairs = rmat27_host
    for pieces in (0, 3):
        sess = skp.HostSession(g.n, g.nnz, pieces=pieces)
        try:
            m_host = sess.run(h_off, h_nb, status_bits=8)
            assert sess.last_mode == "host_mapped" and sess.last_pieces == pieces
            with skp.Graph(g.offsets, g.nbrs, check=False) as h:
                v = h.validate(m_host.cuda())
            m = m_host.numpy().view(np.uint32)
            _oracle_agrees(off, nb, m, v, sgmm_pairs)
            assert _check_sampled_vertices(g, m, 100_000, seed=7 + pieces) > 0
        finally:
            sess.close()


def test_edge_list_rmat27_raw_draws_in_the_benchmark_launch(skp, rmat27, rmat27_host):
    """The 2^31 generator draws behind the CSR, as a list (repeats and loops
    kept, no symmetrisation).  Its edge set, loops aside, is the CSR's, so the
    oracle's CSR checker decides the verdict over the whole graph (the list
    checker sorts the 2^31 list keys on one core, about ten minutes); for a
    valid result the two checkers' verdicts coincide field by field, and the
    device's list checker must give that verdict too."""
    g = rmat27
    _, _, off, nb, sgmm_pairs = rmat27_host
    src, dst = gg.rmat_edges(SCALE, EF << SCALE, .57, .19, .19, 1, "cuda")
    try:
        with skp.EdgeList(g.n, src, dst, check=False) as h:
            mate = h.skipper(**BENCH_COO_OPTS)
            v = h.validate(mate)
        m = mate.cpu().numpy().view(np.uint32)
        _oracle_agrees(off, nb, m, v, sgmm_pairs)
        assert _check_sampled_vertices(g, m, 200_000, seed=4) > 0
        rng = np.random.default_rng(5)
        i = torch.from_numpy(rng.integers(0, src.numel(), 2_000_000)).cuda()
        xs, ys = src[i].cpu().numpy().view(np.uint32), dst[i].cpu().numpy().view(np.uint32)
        real = xs != ys
        assert np.all((m[xs[real]] != NONE) | (m[ys[real]] != NONE))
    finally:
        del src, dst
        torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def c4_batch():
    """The benchmark's batch: 4096 graphs of 10^3..10^6 undirected edges (ER /
    R-MAT / grid in turn), packed block-diagonally with global ids."""
    packed, _ = gg.batch_packed(4096, 1e3, 1e6, seed=101, device="cuda", chunks=4)
    off = packed.csr.offsets.cpu().numpy()
    nb = packed.csr.nbrs.cpu().numpy()
    vb = packed.vbase.cpu().numpy()
    eb = packed.ebase.cpu().numpy()
    _, sgmm_pairs = oracle.sgmm(off, nb)
    yield packed, off, nb, vb, eb, len(sgmm_pairs)
    del packed
    torch.cuda.empty_cache()


@pytest.mark.parametrize("bits", [8, 2])
def test_batched_4096_graphs_in_the_benchmark_launch(skp, c4_batch, bits):
    """CUDA-graph replays over the whole batch (dispersed and ascending units):
    the union and every member graph (rebased to local ids) are checked by the
    oracle, the batch checker agrees with the union checker, and the device's
    per-graph pair counts equal the oracle's."""
    packed, off, nb, vb, eb, sgmm_pairs = c4_batch
    csr = packed.csr
    with skp.Graph(csr.offsets, csr.nbrs, check=False) as h:
        for rep in range(2):     # the second replay reuses the captured graph
            mate, gp = h.batched(packed.vbase, packed.ebase, graph_pairs=True, use_graph=1,
                                 status_bits=bits, grain=8192, block_threads=512,
                                 unit_order=2 - rep)   # dispersed, then ascending
            v = h.validate(mate)
            m = mate.cpu().numpy().view(np.uint32)
            _oracle_agrees(off, nb, m, v, sgmm_pairs)
            assert h.validate_batched(packed.vbase, packed.ebase, mate).as_dict() == v.as_dict()
    gp = gp.cpu().numpy()
    G = vb.size - 1
    for k in range(G):
        lo, hi, e0, e1 = int(vb[k]), int(vb[k + 1]), int(eb[k]), int(eb[k + 1])
        loc = m[lo:hi].astype(np.int64)
        loc = np.where(loc == NONE, NONE, loc - lo).astype(np.uint32)
        vk = oracle.check(off[lo:hi + 1] - e0, (nb[e0:e1].astype(np.int64) - lo).astype(np.uint32), loc)
        assert vk.flags == 0, (k, vk.as_dict())
        assert int(gp[k]) == vk.n_pairs, k
