"""Batched Skipper (block-diagonal packing, one persistent launch, CUDA graph)
against the oracle and against one launch per graph."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from tests.conftest import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

NONE = 0xFFFFFFFF


@pytest.fixture(scope="module")
def skp():
    import paper_2507_04420_gb300 as m
    torch.cuda.set_device(0)
    return m


@pytest.fixture(scope="module")
def batch():
    graphs = gg.batch_mix(48, 1e2, 3e4, seed=21)
    packed = gg.pack(graphs)
    return graphs, packed


def _np(t):
    return t.cpu().numpy().view(np.uint32)


def _local(m, lo, hi):
    s = m[lo:hi].astype(np.int64)
    return np.where(s == NONE, NONE, s - lo).astype(np.uint32)


def test_batched_serial_equals_sgmm_per_graph(skp, batch):
    graphs, packed = batch
    d = packed.csr.to("cuda")
    vb, eb = packed.vbase.cuda(), packed.ebase.cuda()
    off, nb = packed.csr.offsets.numpy(), packed.csr.nbrs.numpy()
    ref_union, _ = oracle.sgmm(off, nb)
    with skp.Graph(d.offsets, d.nbrs) as h:
        for bits in (2, 8, 32):
            for use_graph in (0, 1):
                mate, gp = h.batched(vb, eb, graph_pairs=True, serial=1, status_bits=bits,
                                     use_graph=use_graph)
                m = _np(mate)
                assert np.array_equal(m, ref_union)
                for k, g in enumerate(graphs):
                    lo, hi = int(packed.vbase[k]), int(packed.vbase[k + 1])
                    ref, ref_pairs = oracle.sgmm(g.offsets.numpy(), g.nbrs.numpy())
                    assert np.array_equal(_local(m, lo, hi), ref)          # alone == in the mix
                    assert int(gp[k]) == len(ref_pairs)


@pytest.mark.parametrize("bits", [2, 8, 32])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_batched_parallel_valid(skp, batch, bits, use_graph):
    graphs, packed = batch
    d = packed.csr.to("cuda")
    vb, eb = packed.vbase.cuda(), packed.ebase.cuda()
    off, nb = packed.csr.offsets.numpy(), packed.csr.nbrs.numpy()
    with skp.Graph(d.offsets, d.nbrs) as h:
        for rep in range(3):   # graph replays with a fresh output buffer each time
            mate, gp = h.batched(vb, eb, graph_pairs=True, status_bits=bits, use_graph=use_graph,
                                 grain=128 * (1 + rep))
            m = _np(mate)
            vr = oracle.check(off, nb, m)
            vd = h.validate(mate)
            assert vr.flags == 0 and vd.as_dict() == vr.as_dict()
            for k, g in enumerate(graphs):
                lo, hi = int(packed.vbase[k]), int(packed.vbase[k + 1])
                ml = _local(m, lo, hi)
                v = oracle.check(g.offsets.numpy(), g.nbrs.numpy(), ml)
                assert v.flags == 0
                assert int(gp[k]) == v.n_pairs


def test_each_graph_alone_and_in_the_mix(skp, batch):
    graphs, packed = batch
    d = packed.csr.to("cuda")
    vb, eb = packed.vbase.cuda(), packed.ebase.cuda()
    with skp.Graph(d.offsets, d.nbrs) as h:
        mix = _np(h.batched(vb, eb))
    for k in (0, 1, 2, 17, 47):
        g = graphs[k]
        gd = g.to("cuda")
        with skp.Graph(gd.offsets, gd.nbrs) as hg:
            alone = _np(hg.skipper())
        lo, hi = int(packed.vbase[k]), int(packed.vbase[k + 1])
        off, nb = g.offsets.numpy(), g.nbrs.numpy()
        assert oracle.check(off, nb, alone).flags == 0
        assert oracle.check(off, nb, _local(mix, lo, hi)).flags == 0


def test_autotune_picks_a_valid_setting(skp, batch):
    _, packed = batch
    d = packed.csr.to("cuda")
    vb, eb = packed.vbase.cuda(), packed.ebase.cuda()
    with skp.Graph(d.offsets, d.nbrs) as h:
        o = h.autotune_batched(vb, eb)
        assert o.status_bits in (2, 8, 32) and o.grain in (1024, 2048, 4096, 8192)
        mate = h.batched(vb, eb, opts=o)
        assert h.validate(mate).flags == 0
