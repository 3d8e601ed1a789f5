"""mm_skipper_to_host: the pass in ascending launches with each finished
prefix of the mate array copied into page-locked host memory while later
launches run.  The host copy must equal the device result element for
element (a prefix copied before its rows were finished would differ), the
result must pass the oracle's checker, serial-equivalent settings are not
needed for that, and what the call does not run is refused with a reason."""
import ctypes

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


def _graphs():
    iso = gg.CSR(torch.tensor([0, 0, 2, 2, 4, 4, 4], dtype=torch.int64),
                 torch.tensor([3, 3, 1, 1], dtype=torch.int32))          # rows 0, 2, 5 empty; repeats
    return [("rmat14", gg.rmat(14, 16, seed=5)), ("star", gg.star(200_000)), ("path", gg.path(50_001)),
            ("grid", gg.grid(300, 301)), ("er", gg.erdos_renyi(20_000, 90_000, seed=6)),
            ("isolated", iso), ("one", gg.path(1)), ("two", gg.path(2))]


def _pinned_empty(n):
    return torch.empty(n, dtype=torch.int32, pin_memory=True)


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_host_copy_equals_device_result_and_is_valid(skp, bits):
    for name, g in _graphs():
        off, nb = g.offsets.numpy(), g.nbrs.numpy()
        with skp.Graph(g.offsets.cuda(), g.nbrs.cuda(), check=True) as h:
            for pieces in (1, 2, 3, 8, 64):
                for grain in (128, 2048):
                    hm = _pinned_empty(g.n)
                    hm.fill_(7)
                    dm = torch.full((g.n,), 5, dtype=torch.int32, device="cuda")
                    h.skipper_to_host(hm, mate=dm, pieces=pieces, status_bits=bits, grain=grain)
                    assert torch.equal(hm, dm.cpu()), (name, pieces, grain)
                    assert h.validate(dm).flags == 0, (name, pieces, grain)
                    assert oracle.check(off, nb, hm.numpy().view(np.uint32)).flags == 0, (name, pieces)


def test_read_in_place_with_both_register_budgets(skp):
    g = gg.rmat(15, 16, seed=8)
    off, nb = g.offsets.numpy(), g.nbrs.numpy()
    with skp.Graph(g.offsets.pin_memory(), g.nbrs.pin_memory(), check=False, host_mapped=True) as h:
        for bps in (0, 3, 4):
            for pieces in (4, 16):
                hm = _pinned_empty(g.n)
                dm = torch.empty(g.n, dtype=torch.int32, device="cuda")
                h.skipper_to_host(hm, mate=dm, pieces=pieces, status_bits=8, grain=2048, blocks_per_sm=bps)
                assert torch.equal(hm, dm.cpu())
                assert oracle.check(off, nb, hm.numpy().view(np.uint32)).flags == 0


@pytest.mark.parametrize("kw", [dict(symmetric=1), dict(id_loads=2), dict(l2_persist=1),
                                dict(status_bits=2, blocks_per_sm=3), dict(unit_order=1, grain=384)])
def test_options_the_pass_keeps(skp, kw):
    """Options that change how the sweep runs but not the ascending launches."""
    for g in (gg.rmat(15, 16, seed=12), gg.grid(200, 257), gg.star(30_000)):
        off, nb = g.offsets.numpy(), g.nbrs.numpy()
        with skp.Graph(g.offsets.cuda(), g.nbrs.cuda()) as h:
            hm = _pinned_empty(g.n)
            dm = torch.empty(g.n, dtype=torch.int32, device="cuda")
            h.skipper_to_host(hm, mate=dm, pieces=5, **kw)
            assert torch.equal(hm, dm.cpu()), kw
            assert oracle.check(off, nb, hm.numpy().view(np.uint32)).flags == 0, kw


def test_a_packed_batch_with_global_ids(skp):
    """A block-diagonal batch is one CSR to this call; every member graph's
    part of the host copy is a maximal matching of that graph."""
    packed, _ = gg.batch_packed(24, 1e3, 3e4, seed=13, device="cuda")
    csr = packed.csr
    with skp.Graph(csr.offsets, csr.nbrs) as h:
        hm = _pinned_empty(csr.n)
        dm = torch.empty(csr.n, dtype=torch.int32, device="cuda")
        h.skipper_to_host(hm, mate=dm, pieces=7)
        assert torch.equal(hm, dm.cpu())
        assert h.validate_batched(packed.vbase, packed.ebase, dm).flags == 0
    m = hm.numpy().view(np.uint32)
    vb, eb = packed.vbase.cpu().numpy(), packed.ebase.cpu().numpy()
    off, nb = csr.offsets.cpu().numpy(), csr.nbrs.cpu().numpy()
    for k in range(len(vb) - 1):
        v0, v1, e0, e1 = vb[k], vb[k + 1], eb[k], eb[k + 1]
        sub = m[v0:v1].copy()
        sub[sub != 0xFFFFFFFF] -= np.uint32(v0)
        assert oracle.check(off[v0:v1 + 1] - e0, nb[e0:e1] - v0, sub).flags == 0, k


def test_nosync_then_sync(skp):
    g = gg.rmat(13, 16, seed=9)
    with skp.Graph(g.offsets.cuda(), g.nbrs.cuda()) as h:
        hm = _pinned_empty(g.n)
        dm = torch.empty(g.n, dtype=torch.int32, device="cuda")
        h.skipper_to_host(hm, mate=dm, pieces=8, nosync=1)
        h.sync()
        torch.cuda.synchronize()
        assert torch.equal(hm, dm.cpu())
        assert oracle.check(g.offsets.numpy(), g.nbrs.numpy(), hm.numpy().view(np.uint32)).flags == 0


def test_host_session_reads_in_place_and_copies_back_in_pieces(skp):
    g = gg.rmat(14, 16, seed=10)
    sess = skp.HostSession(g.n, g.nnz, pieces=8)
    try:
        m = sess.run(g.offsets.pin_memory(), g.nbrs.pin_memory())
        assert sess.last_mode == "host_mapped" and sess.last_pieces == 8
        assert oracle.check(g.offsets.numpy(), g.nbrs.numpy(), m.numpy().view(np.uint32)).flags == 0
        m2 = sess.run(g.offsets.pin_memory(), g.nbrs.pin_memory(), unit_order=2)   # not with pieces
        assert sess.last_mode == "host_mapped" and sess.last_pieces == 0
        assert oracle.check(g.offsets.numpy(), g.nbrs.numpy(), m2.numpy().view(np.uint32)).flags == 0
    finally:
        sess.close()


def test_refusals_say_why(skp):
    lib = skp.lib
    g = gg.rmat(10, 8, seed=11)
    with skp.Graph(g.offsets.cuda(), g.nbrs.cuda()) as h:
        dm = torch.empty(g.n, dtype=torch.int32, device="cuda")
        hm = _pinned_empty(g.n)

        def call(o, host=hm, pieces=4, mate=dm):
            return lib.mm_skipper_to_host(h._h, ctypes.byref(o), ctypes.c_void_p(mate.data_ptr()),
                                          ctypes.c_void_p(host.data_ptr()), pieces, None)

        for kw in (dict(unit_order=2), dict(stats=1), dict(serial=1), dict(timing=1), dict(use_graph=1)):
            assert call(skp.options(**kw)) == 6, kw          # MM_ERR_UNSUPPORTED
        o = skp.options()
        assert call(o, pieces=0) == 1 and b"pieces" in lib.mm_last_error()
        assert call(o, pieces=65) == 1
        pageable = torch.empty(g.n, dtype=torch.int32)
        assert call(o, host=pageable) == 1 and b"page-locked" in lib.mm_last_error()
        assert call(o, host=dm) == 1                          # device memory is not host memory
        assert lib.mm_skipper_to_host(h._h, ctypes.byref(o), None, ctypes.c_void_p(hm.data_ptr()), 4, None) == 1
        assert call(o) == 0                                   # the handle still works
        torch.cuda.synchronize()
        assert torch.equal(hm, dm.cpu())
    src = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    dst = torch.tensor([1, 2], dtype=torch.int32, device="cuda")
    with skp.EdgeList(3, src, dst) as e:
        dm = torch.empty(3, dtype=torch.int32, device="cuda")
        hm = _pinned_empty(3)
        o = skp.options()
        assert lib.mm_skipper_to_host(e._h, ctypes.byref(o), ctypes.c_void_p(dm.data_ptr()),
                                      ctypes.c_void_p(hm.data_ptr()), 2, None) == 6
