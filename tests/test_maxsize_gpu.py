"""Maximum sizes: n = MM_MAX_VERTICES = 0xFFFFFFFD vertices (the largest id,
0xFFFFFFFC, sits just below the 32-bit state layout's RSVD and ACC words and
the unmatched sentinel), and a multi-graph launch whose total vertex count
exceeds 2^32 (each graph keeps local uint32 ids; states live at 64-bit bases).

The edges touch a few thousand vertices spread over the whole id range, so
the oracle runs on an order-preserving relabelling of the touched vertices:
SGMM visits rows in ascending id and neighbours in stored order, so its result
on the relabelled graph maps back exactly, and every untouched vertex must be
unmatched.  One-thread modes are checked through the edge-list path (the list
in CSR row order equals SGMM), since a single thread walking 4.3G rows would
take minutes.
"""
import numpy as np
import pytest
import torch

import oracle
from tests.conftest import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

NONE = 0xFFFFFFFF
NMAX = 0xFFFFFFFD


@pytest.fixture(scope="module")
def skp():
    import paper_2507_04420_gb300 as m
    torch.cuda.set_device(0)
    return m


def _edges(n, seed):
    """Undirected edges over ids spread across [0, n): a path over the top 600
    ids, a star on the top id, edges between the lowest and highest ids, and
    random pairs among 2000 ids scattered over the range."""
    rng = np.random.default_rng(seed)
    top = np.arange(n - 600, n, dtype=np.int64)
    e = [np.stack([top[:-1], top[1:]], 1)]
    e.append(np.stack([np.full(300, n - 1), rng.choice(np.arange(n - 5000, n - 1), 300, replace=False)], 1))
    e.append(np.array([[0, n - 1], [1, n - 2], [2, n - 3], [3, 4], [n // 2, n - 1]], dtype=np.int64))
    pts = np.unique(rng.integers(0, n, 2000))
    pairs = rng.choice(pts, size=(3000, 2))
    e.append(pairs[pairs[:, 0] != pairs[:, 1]])
    e = np.concatenate(e)
    e = np.unique(np.sort(e, 1), axis=0)
    return e


def _csr_on_device(n, e):
    """Symmetric CSR with rows sorted: offsets filled segment by segment on the
    device (the rows with entries are few), neighbour ids uint32."""
    s = np.concatenate([e[:, 0], e[:, 1]])
    d = np.concatenate([e[:, 1], e[:, 0]])
    order = np.lexsort((d, s))
    s, d = s[order], d[order]
    rows, counts = np.unique(s, return_counts=True)
    offsets = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    prev, acc = 0, 0
    for r, c in zip(rows.tolist(), counts.tolist()):
        offsets[prev:r + 1].fill_(acc)
        acc += c
        prev = r + 1
    offsets[prev:].fill_(acc)
    nbrs = torch.from_numpy(d.astype(np.uint32).view(np.int32)).cuda()
    return offsets, nbrs, s, d


def _relabel(s, d):
    ids = np.unique(np.concatenate([s, d]))
    return ids, np.searchsorted(ids, s), np.searchsorted(ids, d)


def _small_csr(k, s, d):
    off = np.zeros(k + 1, dtype=np.int64)
    np.add.at(off, s + 1, 1)
    return np.cumsum(off), d.astype(np.uint32)


def _touched_mate(mate, ids):
    """mate of the touched vertices, relabelled; and the count of matched
    vertices elsewhere (must be 0)."""
    idx = torch.from_numpy(ids).cuda()
    m = mate[idx].cpu().numpy().view(np.uint32).astype(np.int64)
    others = int((mate != -1).sum()) - int((m != NONE).sum())
    lab = np.full(m.shape, NONE, dtype=np.int64)
    ok = m != NONE
    pos = np.searchsorted(ids, m[ok])
    pos = np.minimum(pos, len(ids) - 1)
    lab[ok] = np.where(ids[pos] == m[ok], pos, NONE - 1)   # a partner outside the touched set: invalid
    return lab.astype(np.uint32), others


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_csr_at_the_largest_n(skp, bits):
    e = _edges(NMAX, seed=1)
    offsets, nbrs, s, d = _csr_on_device(NMAX, e)
    ids, ls, ld = _relabel(s, d)
    off_small, nb_small = _small_csr(len(ids), ls, ld)
    try:
        with skp.Graph(offsets, nbrs, check=True) as h:
            mate, pairs, cnt = h.skipper(status_bits=bits, grain=2048, pairs=True, cap=20000)
            vd = h.validate(mate, pairs[:int(cnt.item())])
        m_small, others = _touched_mate(mate, ids)
        assert others == 0
        vr = oracle.check(off_small, nb_small, m_small)
        assert vr.flags == 0, vr.as_dict()
        assert vd.flags == 0 and vd.n_pairs == vr.n_pairs and vd.n_matched == vr.n_matched
        assert int(cnt.item()) == vr.n_pairs
        p = pairs[:int(cnt.item())].cpu().numpy().view(np.uint32).astype(np.int64)
        assert np.all(p[:, 0] < p[:, 1]) and np.all(np.diff(p[:, 0]) > 0)
    finally:
        del offsets, nbrs
        torch.cuda.empty_cache()


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_edge_list_at_the_largest_n_serial_is_sgmm(skp, bits):
    e = _edges(NMAX, seed=2)
    s = np.concatenate([e[:, 0], e[:, 1]])
    d = np.concatenate([e[:, 1], e[:, 0]])
    order = np.lexsort((d, s))
    s, d = s[order], d[order]          # the symmetric CSR's entries in row order
    ids, ls, ld = _relabel(s, d)
    off_small, nb_small = _small_csr(len(ids), ls, ld)
    ref, _ = oracle.sgmm(off_small, nb_small)
    ds = torch.from_numpy(s.astype(np.uint32).view(np.int32)).cuda()
    dd = torch.from_numpy(d.astype(np.uint32).view(np.int32)).cuda()
    with skp.EdgeList(NMAX, ds, dd) as h:
        mate = h.skipper(status_bits=bits, serial=1)
        m_small, others = _touched_mate(mate, ids)
        assert others == 0 and np.array_equal(m_small, ref)
        mate = h.skipper(status_bits=bits)
        m_small, others = _touched_mate(mate, ids)
        assert others == 0
        vd = h.validate(mate)
        vr = oracle.check(off_small, nb_small, m_small)
        assert vr.flags == 0 and vd.flags == 0 and vd.n_pairs == vr.n_pairs
    del mate
    torch.cuda.empty_cache()


def test_multi_graph_launch_beyond_2_32_vertices(skp):
    n = (1 << 31) + 7                  # two graphs: 2^32 + 14 vertices in one launch
    graphs, smalls = [], []
    try:
        for seed in (3, 4):
            e = _edges(n, seed)
            offsets, nbrs, s, d = _csr_on_device(n, e)
            ids, ls, ld = _relabel(s, d)
            mate = torch.empty(n, dtype=torch.int32, device="cuda")
            graphs.append((offsets, nbrs, mate))
            smalls.append((ids, *_small_csr(len(ids), ls, ld)))
        m = skp.Multi()
        try:
            m.run(graphs, status_bits=8)
            verdicts = m.validate(graphs)
        finally:
            m.close()
        for (off, nb, mate), (ids, off_s, nb_s), vd in zip(graphs, smalls, verdicts):
            m_small, others = _touched_mate(mate, ids)
            assert others == 0
            vr = oracle.check(off_s, nb_s, m_small)
            assert vr.flags == 0 and vd.flags == 0 and vd.n_pairs == vr.n_pairs
    finally:
        del graphs
        torch.cuda.empty_cache()
