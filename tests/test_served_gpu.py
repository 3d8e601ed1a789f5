"""Multi-graph launches and the continuous-batching server against the oracle.

The server matches whatever requests have arrived in one launch while earlier
ones may still be on the GPU.  A request's result must not depend on its
company: in serial mode (one thread per graph, SGMM order) the mate array must
equal the graph's matching computed alone byte for byte; in parallel mode each
result must be a maximal matching that the oracle and the device checker both
accept with identical verdicts.
"""
import threading
import time

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from tests.conftest import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def skp():
    import paper_2507_04420_gb300 as m
    torch.cuda.set_device(0)
    return m


@pytest.fixture(scope="module")
def graphs():
    gs = gg.batch_mix(24, 1e2, 5e4, seed=31)
    gs.append(gg.CSR(torch.zeros(4, dtype=torch.int64), torch.zeros(0, dtype=torch.int32)))  # no edges
    gs.append(gg.star(3000))
    return gs


def _np(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_multi_serial_equals_sgmm_and_parallel_valid(skp, graphs, bits):
    dev = [g.to("cuda") for g in graphs]
    m = skp.Multi()
    try:
        mates = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in graphs]
        tri = [(d.offsets, d.nbrs, mt) for d, mt in zip(dev, mates)]
        m.run(tri, serial=1, status_bits=bits)
        for g, mt in zip(graphs, mates):
            ref, _ = oracle.sgmm(g.offsets.numpy(), g.nbrs.numpy())
            assert np.array_equal(_np(mt), ref)
        for grain, id_loads in ((128, 0), (2048, 0), (128, 2), (2048, 2)):   # eager, selective
            m.run(tri, status_bits=bits, grain=grain, id_loads=id_loads)
            verdicts = m.validate(tri)
            for g, mt, vd in zip(graphs, mates, verdicts):
                vr = oracle.check(g.offsets.numpy(), g.nbrs.numpy(), _np(mt))
                assert vr.flags == 0 and vd.as_dict() == vr.as_dict()
    finally:
        m.close()


def test_multi_validate_reports_corruption_per_graph(skp, graphs):
    dev = [g.to("cuda") for g in graphs[:6]]
    m = skp.Multi()
    try:
        mates = [torch.empty(d.n, dtype=torch.int32, device="cuda") for d in dev]
        tri = [(d.offsets, d.nbrs, mt) for d, mt in zip(dev, mates)]
        m.run(tri)
        mates[3][:] = -1                      # graph 3 left unmatched
        verdicts = m.validate(tri)
        m.validate_async(tri)                 # the enqueued form gives the same verdicts
        torch.cuda.synchronize()
        assert [v.as_dict() for v in m.verdicts(len(tri))] == [v.as_dict() for v in verdicts]
        for k, (g, mt, vd) in enumerate(zip(graphs[:6], mates, verdicts)):
            vr = oracle.check(g.offsets.numpy(), g.nbrs.numpy(), _np(mt))
            assert vd.as_dict() == vr.as_dict()
            assert (vr.flags != 0) == (k == 3 and g.nnz > 0)
    finally:
        m.close()


def _pinned(g):
    return g.offsets.pin_memory(), g.nbrs.pin_memory()


@pytest.mark.parametrize("in_place_max_nnz", [0, 20000, 1 << 20])   # all copied, mixed, all in place
@pytest.mark.parametrize("serial", [1, 0])
def test_server_results_same_alone_and_in_the_mix(skp, graphs, serial, in_place_max_nnz):
    from paper_2507_04420_gb300.server import Server
    alone = []
    for g in graphs:
        d = g.to("cuda")
        with skp.Graph(d.offsets, d.nbrs) as h:
            alone.append(_np(h.skipper(serial=serial, status_bits=32)))
    # a small memory budget forces several admission rounds, and staggered
    # submissions make requests join while earlier ones are on the GPU
    budget = max(4 * 1024 * 1024, 3 * max(g.nnz * 4 + g.n * 12 for g in graphs))
    srv = Server(memory_bytes=budget, serial=bool(serial), status_bits=32,
                 in_place_max_nnz=in_place_max_nnz)
    reqs = []

    def client():
        for rep in range(3):
            for g in graphs:
                reqs.append((g, srv.submit(*_pinned(g))))
                if len(reqs) % 7 == 0:
                    time.sleep(0.002)

    t = threading.Thread(target=client)
    t.start()
    t.join()
    for _, r in reqs:
        assert r.wait(120)
    srv.close()
    assert srv.ticks > 1
    assert all(r.in_place == (g.nnz <= in_place_max_nnz) for g, r in reqs)
    for idx, (g, r) in enumerate(reqs):
        assert r.error is None
        m = r.mate.numpy().view(np.uint32)
        vr = oracle.check(g.offsets.numpy(), g.nbrs.numpy(), m)
        assert vr.flags == 0 and r.verdict.as_dict() == vr.as_dict()
        if serial:
            assert np.array_equal(m, alone[idx % len(graphs)])
        assert r.latency is not None and r.latency > 0


def test_server_rejects_what_can_never_fit(skp):
    from paper_2507_04420_gb300.server import Server, device_bytes
    g = gg.rmat(14, 16, seed=2)
    assert device_bytes(g.n, g.nnz) > (1 << 20) > device_bytes(g.n, g.nnz, in_place=True)
    srv = Server(memory_bytes=1 << 20, in_place_max_nnz=0)   # every request copied
    r = srv.submit(*_pinned(g))
    assert r.wait(5) and isinstance(r.error, MemoryError)
    small = gg.path(100)
    r2 = srv.submit(*_pinned(small))
    assert r2.wait(60) and r2.error is None and r2.verdict.flags == 0
    srv.close()
    srv = Server(memory_bytes=1 << 20)                       # read in place, the CSR stays on the host
    r3 = srv.submit(*_pinned(g))
    assert r3.wait(60) and r3.error is None and r3.in_place and r3.verdict.flags == 0
    vr = oracle.check(g.offsets.numpy(), g.nbrs.numpy(), r3.mate.numpy().view(np.uint32))
    assert vr.flags == 0 and vr.as_dict() == r3.verdict.as_dict()
    srv.close()


def test_server_many_client_threads(skp, graphs):
    """Four client threads submit at once; every result matches the graph's
    serial result alone (SGMM order), whichever way the request went in."""
    from paper_2507_04420_gb300.server import Server
    alone = {}
    for i, g in enumerate(graphs):
        ref, _ = oracle.sgmm(g.offsets.numpy(), g.nbrs.numpy())
        alone[i] = ref
    pinned = [_pinned(g) for g in graphs]
    srv = Server(serial=True, status_bits=8, in_place_max_nnz=20000)
    out = [[] for _ in range(4)]

    def client(k):
        for rep in range(3):
            for i in range(k, len(graphs), 2):
                out[k].append((i, srv.submit(*pinned[i])))

    ts = [threading.Thread(target=client, args=(k,)) for k in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for lst in out:
        for i, r in lst:
            assert r.wait(120) and r.error is None
            assert np.array_equal(r.mate.numpy().view(np.uint32), alone[i])
            assert r.verdict.flags == 0 and r.latency >= 0
    srv.close()
    assert srv.ticks >= 1 and srv.graphs_launched == sum(len(x) for x in out)


def test_server_worker_failure_fails_requests_and_frees_device_memory(skp):
    """A device allocation that fails inside the worker ends the serving loop
    cleanly: the request fails with MM_ERR_OOM, later submits are refused,
    destroy reports the failure, and the buffer already allocated for the
    request is released.  The request is a copy-path graph of 2^31 - 1 vertices
    and 2^40 entries, admitted under a budget that claims 2^62 bytes: its 16 GiB
    of offsets are allocated, its 4 TiB neighbour array cannot be, and no copy
    or kernel runs (the copies follow the three allocations), so the small
    host arrays passed are never read."""
    import ctypes
    from paper_2507_04420_gb300 import lib
    from paper_2507_04420_gb300._native import ServerConfig, ServerResult
    MM_ERR_OOM = 2

    def ptr(t):
        return ctypes.c_void_p(t.data_ptr())

    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    cfg = ServerConfig()
    assert lib.mm_server_default_config(ctypes.byref(cfg)) == 0
    cfg.memory_bytes = 1 << 62
    cfg.in_place_max_nnz = 0
    h = ctypes.c_void_p()
    assert lib.mm_server_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    off = torch.zeros(2, dtype=torch.int64)
    nb = torch.zeros(4, dtype=torch.int32)
    mate = torch.zeros(4, dtype=torch.int32)
    t = ctypes.c_uint64()
    assert lib.mm_server_submit(h, (1 << 31) - 1, 1 << 40, ptr(off), ptr(nb), ptr(mate), ctypes.byref(t)) == 0
    res = ServerResult()
    assert lib.mm_server_wait(h, t.value, 120.0, ctypes.byref(res)) == 0
    assert res.status == MM_ERR_OOM and res.in_place == 0
    t2 = ctypes.c_uint64()
    assert lib.mm_server_submit(h, 1, 0, ptr(off), None, ptr(mate), ctypes.byref(t2)) == MM_ERR_OOM
    assert lib.mm_server_destroy(h) == MM_ERR_OOM
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (1 << 30), (free0, free1)   # the 16 GiB came back
