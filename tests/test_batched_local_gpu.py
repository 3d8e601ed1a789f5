"""Batched Skipper with a partition per member graph: local ids
(MM_BATCH_LOCAL_IDS), the warps-per-graph cap, the batch checker
(mm_validate_batched), and a batch of more than 2^32 vertices in one CUDA-graph
replay -- every member graph checked by the oracle (Section II-B), serial mode
equal to SGMM graph by graph."""
import ctypes

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from tests.conftest import cuda_ok
from tests.test_maxsize_gpu import _csr_on_device, _edges, _relabel, _small_csr, _touched_mate

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

NONE = 0xFFFFFFFF
U64MAX = (1 << 64) - 1
FIELDS = ("flags", "n_matched", "n_pairs", "n_bad_range", "n_asym", "n_nonedge", "n_uncovered",
          "n_pairs_bad", "first_bad_vertex", "first_uncovered")


@pytest.fixture(scope="module")
def skp():
    import paper_2507_04420_gb300 as m
    torch.cuda.set_device(0)
    return m


@pytest.fixture(scope="module")
def batch():
    graphs = gg.batch_mix(48, 1e2, 3e4, seed=31)
    # a graph with no vertex and one with vertices but no entry, between the others
    graphs.insert(5, gg.CSR(torch.zeros(1, dtype=torch.int64), torch.zeros(0, dtype=torch.int32)))
    graphs.insert(9, gg.CSR(torch.zeros(8, dtype=torch.int64), torch.zeros(0, dtype=torch.int32)))
    return graphs, gg.pack(graphs, local=True), gg.pack(graphs)


def _np(t):
    return t.cpu().numpy().view(np.uint32)


def _union_oracle(graphs, packed, m, local):
    """The oracle's verdict on every member graph, summed as one batch verdict."""
    vb, eb = packed.vbase.cpu().numpy(), packed.ebase.cpu().numpy()
    u = dict.fromkeys(FIELDS, 0)
    u["first_bad_vertex"] = u["first_uncovered"] = U64MAX
    per = []
    for k, g in enumerate(graphs):
        lo, hi = int(vb[k]), int(vb[k + 1])
        ml = m[lo:hi].astype(np.int64)
        if not local:
            ml = np.where(ml == NONE, NONE, ml - lo)
        v = oracle.check(g.offsets.numpy(), g.nbrs.numpy(), ml.astype(np.uint32))
        per.append(v)
        d = v.as_dict()
        for f in FIELDS[1:8]:
            u[f] += d[f]
        u["flags"] |= d["flags"]
        if d["first_bad_vertex"] != U64MAX:
            u["first_bad_vertex"] = min(u["first_bad_vertex"], lo + d["first_bad_vertex"])
        if d["first_uncovered"] != U64MAX:
            u["first_uncovered"] = min(u["first_uncovered"], int(eb[k]) + d["first_uncovered"])
    return u, per


def test_serial_local_ids_equal_sgmm_per_graph(skp, batch):
    graphs, packed, _ = batch
    d = packed.csr.to("cuda")
    vb, eb = packed.vbase.cuda(), packed.ebase.cuda()
    refs = [oracle.sgmm(g.offsets.numpy(), g.nbrs.numpy()) for g in graphs]
    with skp.Graph(d.offsets, d.nbrs, check=False, local_ids=True) as h:
        for bits in (2, 8, 32):
            for use_graph in (0, 1):
                for rep in range(2):
                    mate, gp = h.batched(vb, eb, graph_pairs=True, serial=1, status_bits=bits,
                                         use_graph=use_graph)
                    m = _np(mate)
                    for k, (ref, ref_pairs) in enumerate(refs):
                        lo, hi = int(packed.vbase[k]), int(packed.vbase[k + 1])
                        assert np.array_equal(m[lo:hi], ref), (bits, use_graph, k)
                        assert int(gp[k]) == len(ref_pairs)


@pytest.mark.parametrize("bits", [2, 8, 32])
@pytest.mark.parametrize("use_graph", [0, 1])
@pytest.mark.parametrize("wpg", [0, 1, 3])
def test_parallel_local_ids_valid_per_graph(skp, batch, bits, use_graph, wpg):
    graphs, packed, _ = batch
    d = packed.csr.to("cuda")
    vb, eb = packed.vbase.cuda(), packed.ebase.cuda()
    with skp.Graph(d.offsets, d.nbrs, check=False, local_ids=True) as h:
        for grain, order in ((128, 1), (1024, 2), (128, 0)):
            mate, gp = h.batched(vb, eb, graph_pairs=True, status_bits=bits, use_graph=use_graph,
                                 warps_per_graph=wpg, grain=grain, unit_order=order)
            m = _np(mate)
            u, per = _union_oracle(graphs, packed, m, local=True)
            assert u["flags"] == 0, u
            assert h.validate_batched(vb, eb, mate).as_dict() == u
            assert [int(x) for x in gp.cpu()] == [v.n_pairs for v in per]


@pytest.mark.parametrize("wpg", [1, 2, 64])
def test_global_ids_with_a_warp_cap(skp, batch, wpg):
    """Global ids, every graph split on its own: valid on the union and per
    graph; the batch checker equals mm_validate field by field."""
    graphs, _, packed = batch
    d = packed.csr.to("cuda")
    vb, eb = packed.vbase.cuda(), packed.ebase.cuda()
    off, nb = packed.csr.offsets.numpy(), packed.csr.nbrs.numpy()
    with skp.Graph(d.offsets, d.nbrs) as h:
        for bits, order in ((2, 0), (8, 2), (32, 1)):
            mate, gp = h.batched(vb, eb, graph_pairs=True, status_bits=bits, warps_per_graph=wpg,
                                 grain=128, use_graph=1, unit_order=order)
            m = _np(mate)
            vr = oracle.check(off, nb, m)
            vd = h.validate(mate)
            assert vr.flags == 0 and vd.as_dict() == vr.as_dict()
            assert h.validate_batched(vb, eb, mate).as_dict() == vr.as_dict()
            u, per = _union_oracle(graphs, packed, m, local=False)
            assert [int(x) for x in gp.cpu()] == [v.n_pairs for v in per]
        mate = h.batched(vb, eb, serial=1, warps_per_graph=wpg)
        assert np.array_equal(_np(mate), oracle.sgmm(off, nb)[0])


def test_batch_checker_on_corrupted_results(skp, batch):
    """The batch checker's counts and first offenders equal the oracle's
    (summed over the member graphs) on deliberately broken mate arrays."""
    graphs, packed, _ = batch
    d = packed.csr.to("cuda")
    vb, eb = packed.vbase.cuda(), packed.ebase.cuda()
    with skp.Graph(d.offsets, d.nbrs, check=False, local_ids=True) as h:
        good = _np(h.batched(vb, eb, serial=1))
        vbase = packed.vbase.numpy()
        rng = np.random.default_rng(4)
        cases = []
        for _ in range(12):
            m = good.copy()
            k = int(rng.integers(0, len(graphs)))
            lo, hi = int(vbase[k]), int(vbase[k + 1])
            matched = np.nonzero(m[lo:hi] != NONE)[0]
            if matched.size == 0:
                continue
            v = int(rng.choice(matched))
            w = int(m[lo + v])
            kind = len(cases) % 4
            if kind == 0:        # drop a match: asymmetry, maybe uncovered edges
                m[lo + v] = NONE
            elif kind == 1:      # drop both ends: uncovered edges
                m[lo + v] = NONE
                m[lo + w] = NONE
            elif kind == 2:      # out of the graph's range
                m[lo + v] = hi - lo + 3
            else:                # two pairs (v, w), (x, y) re-paired as (v, x), (w, y): often no edge
                others = [int(a) for a in matched if int(a) not in (v, w)]
                if not others:
                    continue
                x = others[0]
                y = int(m[lo + x])
                m[lo + v], m[lo + x], m[lo + w], m[lo + y] = x, v, y, w
            cases.append(m)
        flagged = 0
        for m in cases:
            t = torch.from_numpy(m.view(np.int32)).cuda()
            u, _ = _union_oracle(graphs, packed, m, local=True)
            flagged += u["flags"] != 0
            assert h.validate_batched(vb, eb, t).as_dict() == u
        assert flagged >= 3


def test_local_id_handle_refuses_single_graph_calls(skp, batch):
    _, packed, _ = batch
    d = packed.csr.to("cuda")
    with skp.Graph(d.offsets, d.nbrs, check=False, local_ids=True) as h:
        with pytest.raises(skp.SkipperError) as e:
            h.skipper()
        assert e.value.code == 6
        with pytest.raises(skp.SkipperError) as e:
            h.validate(torch.empty(d.n, dtype=torch.int32, device="cuda"))
        assert e.value.code == 6
    with pytest.raises(skp.SkipperError) as e:
        skp.Graph(d.offsets, d.nbrs, check=True, local_ids=True)
    assert e.value.code == 6


def test_autotune_on_local_ids(skp, batch):
    graphs, packed, _ = batch
    d = packed.csr.to("cuda")
    vb, eb = packed.vbase.cuda(), packed.ebase.cuda()
    with skp.Graph(d.offsets, d.nbrs, check=False, local_ids=True) as h:
        o = h.autotune_batched(vb, eb)
        assert o.warps_per_graph in (0, 1, 4, 16) and o.grain in (1024, 2048, 4096, 8192)
        o.use_graph = 1
        mate = h.batched(vb, eb, opts=o)
        u, _ = _union_oracle(graphs, packed, _np(mate), local=True)
        assert u["flags"] == 0


def test_local_ids_batch_beyond_2_32_vertices(skp):
    """Two graphs of 2^31 + 7 vertices (2^32 + 14 in the batch), local ids, one
    CUDA-graph replay; each graph checked by the oracle on an order-preserving
    relabelling of its touched vertices (every other vertex stays unmatched)."""
    n = (1 << 31) + 7
    parts, smalls = [], []
    for seed in (5, 6):
        e = _edges(n, seed)
        offsets, nbrs, s, dd = _csr_on_device(n, e)
        parts.append((offsets, nbrs))
        ids, ls, ld = _relabel(s, dd)
        smalls.append((ids, *_small_csr(len(ids), ls, ld)))
    nnz0 = parts[0][1].numel()
    offsets = torch.cat([parts[0][0][:-1], parts[1][0] + nnz0])
    nbrs = torch.cat([parts[0][1], parts[1][1]])
    del parts
    torch.cuda.empty_cache()
    vb = torch.tensor([0, n, 2 * n], dtype=torch.int64, device="cuda")
    eb = torch.tensor([0, nnz0, nbrs.numel()], dtype=torch.int64, device="cuda")
    try:
        with skp.Graph(offsets, nbrs, check=False, local_ids=True) as h:
            for bits in (8, 2):
                mate, gp = h.batched(vb, eb, graph_pairs=True, status_bits=bits, use_graph=1, grain=2048)
                vd = h.validate_batched(vb, eb, mate)
                assert vd.flags == 0, vd.as_dict()
                total = 0
                for k, (ids, off_s, nb_s) in enumerate(smalls):
                    m_small, others = _touched_mate(mate[k * n:(k + 1) * n], ids)
                    assert others == 0
                    vr = oracle.check(off_s, nb_s, m_small)
                    assert vr.flags == 0 and int(gp[k]) == vr.n_pairs
                    total += vr.n_pairs
                assert vd.n_pairs == total
                del mate
    finally:
        del offsets, nbrs
        torch.cuda.empty_cache()
