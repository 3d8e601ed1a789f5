"""Seeded random graphs through random option settings, every result checked
by the oracle (Section II-B's definition) and by the device checker with an
identical verdict: state layout, register budget (blocks per SM), unit order
(ascending or dispersed), grain (0: chosen by the library), symmetric filter,
the result copied to host memory in pieces while the pass runs, and for batches global or
local ids with a warps-per-graph cap, with and without the CUDA graph.  The
graphs mix families and shapes the fixed tests do not pin: loops, unsorted
rows, empty rows, isolated vertices and runs of consecutive ids."""
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


def _random_graph(rng):
    kind = rng.integers(0, 6)
    if kind == 0:
        n = int(rng.integers(1, 3000))
        return gg.erdos_renyi(n, int(rng.integers(0, min(4 * n, n * (n - 1) // 2) + 1)), seed=int(rng.integers(1 << 30)))
    if kind == 1:
        return gg.rmat(int(rng.integers(4, 13)), int(rng.integers(1, 17)), seed=int(rng.integers(1 << 30)))
    if kind == 2:
        return gg.grid(int(rng.integers(1, 80)), int(rng.integers(1, 80)))
    if kind == 3:
        return gg.path(int(rng.integers(1, 5000)))
    if kind == 4:   # loops, repeats and unsorted rows
        n = int(rng.integers(2, 400))
        m = int(rng.integers(0, 4 * n))
        u = rng.integers(0, n, m)
        v = rng.integers(0, n, m)
        s = np.concatenate([u, v])
        d = np.concatenate([v, u])
        order = np.argsort(s, kind="stable")
        s, d = s[order], d[order]
        off = np.zeros(n + 1, dtype=np.int64)
        np.add.at(off, s + 1, 1)
        off = np.cumsum(off)
        for x in range(n):   # shuffle within rows
            a, b = off[x], off[x + 1]
            d[a:b] = rng.permutation(d[a:b])
        return gg.CSR(torch.from_numpy(off), torch.from_numpy(d.astype(np.int32)))
    # many isolated vertices around a few dense rows
    n = int(rng.integers(100, 20000))
    k = int(rng.integers(1, 50))
    hubs = rng.integers(0, n, k)
    u = np.repeat(hubs, 40)
    v = rng.integers(0, n, u.size)
    return gg.from_edges(n, torch.from_numpy(u), torch.from_numpy(v))


def _opts(rng):
    bits = int(rng.choice([2, 8, 32]))
    return dict(status_bits=bits, grain=int(rng.choice([0, 128, 256, 1024, 8192])),
                blocks_per_sm=int(rng.choice([0, 1, 3, 4])), unit_order=int(rng.integers(0, 3)),
                block_threads=int(rng.choice([128, 256, 512])))


def test_random_graphs_and_options(skp):
    rng = np.random.default_rng(2024)
    for it in range(60):
        g = _random_graph(rng)
        o = _opts(rng)
        if o["blocks_per_sm"] * o["block_threads"] > 2048:
            o["blocks_per_sm"] = 0
        off, nb = g.offsets.numpy(), g.nbrs.numpy()
        d = g.to("cuda")
        with skp.Graph(d.offsets, d.nbrs) as h:
            mate = h.skipper(**o)
            m = mate.cpu().numpy().view(np.uint32)
            vr = oracle.check(off, nb, m)
            assert vr.flags == 0, (it, o, vr.as_dict())
            assert h.validate(mate).as_dict() == vr.as_dict(), (it, o)
            if o["unit_order"] != 2:   # the pieces need ascending units
                pieces = int(rng.integers(1, 9))
                hm = torch.empty(g.n, dtype=torch.int32, pin_memory=True)
                h.skipper_to_host(hm, mate=mate, pieces=pieces, **o)
                assert torch.equal(hm, mate.cpu()), (it, o, pieces)
                assert oracle.check(off, nb, hm.numpy().view(np.uint32)).flags == 0, (it, o, pieces)


def test_random_batches_and_options(skp):
    rng = np.random.default_rng(77)
    for it in range(12):
        G = int(rng.integers(1, 40))
        graphs = [_random_graph(rng) for _ in range(G)]
        local = bool(rng.integers(0, 2))
        packed = gg.pack(graphs, local=local)
        o = _opts(rng)
        if o["blocks_per_sm"] * o["block_threads"] > 2048:
            o["blocks_per_sm"] = 0
        o["warps_per_graph"] = int(rng.choice([0, 0, 1, 2, 7]))
        o["use_graph"] = int(rng.integers(0, 2))
        d = packed.csr.to("cuda")
        vb, eb = packed.vbase.cuda(), packed.ebase.cuda()
        with skp.Graph(d.offsets, d.nbrs, check=False, local_ids=local) as h:
            for rep in range(2):
                mate, gp = h.batched(vb, eb, graph_pairs=True, **o)
                m = mate.cpu().numpy().view(np.uint32)
                for k, g in enumerate(graphs):
                    lo, hi = int(packed.vbase[k]), int(packed.vbase[k + 1])
                    ml = m[lo:hi].astype(np.int64)
                    if not local:
                        ml = np.where(ml == NONE, NONE, ml - lo)
                    v = oracle.check(g.offsets.numpy(), g.nbrs.numpy(), ml.astype(np.uint32))
                    assert v.flags == 0, (it, k, o, local, v.as_dict())
                    assert int(gp[k]) == v.n_pairs, (it, k)
                vd = h.validate_batched(vb, eb, mate)
                assert vd.flags == 0, (it, o, local, vd.as_dict())
