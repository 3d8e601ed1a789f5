"""MM_HOST_MAPPED: the kernels read a CSR or an edge list in place from
page-locked host memory.  Same results as from device memory: serial mode
byte-identical to SGMM, parallel verdicts identical to the oracle's; the host
session's zero-copy and copy modes agree; unpinned memory is refused."""
import ctypes

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


def _np(t):
    return t.cpu().numpy().view(np.uint32)


def _pinned(t):
    return t.contiguous().pin_memory()


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_csr_read_in_place(skp, bits):
    for g in (gg.rmat(12, 16, seed=3), gg.grid(40, 50), gg.star(2000), gg.path(1001)):
        off, nb = g.offsets.numpy(), g.nbrs.numpy()
        ref, _ = oracle.sgmm(off, nb)
        with skp.Graph(_pinned(g.offsets), _pinned(g.nbrs), check=True, host_mapped=True) as h:
            assert np.array_equal(_np(h.skipper(status_bits=bits, serial=1)), ref)
            for sym in (0, 1):
                mate, pairs, cnt = h.skipper(status_bits=bits, pairs=True, symmetric=sym, grain=256)
                k = int(cnt.item())
                vr = oracle.check(off, nb, _np(mate), _np(pairs[:k]).reshape(-1, 2))
                vd = h.validate(mate, pairs[:k])
                assert vr.flags == 0 and vd.as_dict() == vr.as_dict()


def test_edge_list_read_in_place(skp):
    g = gg.rmat(12, 8, seed=5)
    s, d = gg.edge_list(g, "shuffle", seed=5)
    src, dst = _np(s), _np(d)
    ref, _ = oracle.sgmm_edges(g.n, src, dst)
    with skp.EdgeList(g.n, _pinned(s), _pinned(d), host_mapped=True) as h:
        for bits in (2, 8, 32):
            assert np.array_equal(_np(h.skipper(status_bits=bits, serial=1)), ref)
            mate = h.skipper(status_bits=bits)
            vr = oracle.check_edges(g.n, src, dst, _np(mate))
            assert vr.flags == 0 and h.validate(mate).as_dict() == vr.as_dict()


def test_host_session_zero_copy_and_copy_agree(skp):
    graphs = [gg.rmat(11, 8, seed=s) for s in (1, 2)] + [gg.erdos_renyi(3000, 9000, seed=3)]
    n_max = max(g.n for g in graphs)
    nnz_max = max(g.nnz for g in graphs)
    zc = skp.HostSession(n_max, nnz_max)
    cp = skp.HostSession(n_max, nnz_max, zero_copy=False)
    try:
        for g in graphs:
            off, nb = _pinned(g.offsets), _pinned(g.nbrs)
            ref, _ = oracle.sgmm(g.offsets.numpy(), g.nbrs.numpy())
            a = zc.run(off, nb, serial=1)
            assert zc.last_mode == "host_mapped"
            b = cp.run(off, nb, serial=1)
            assert cp.last_mode == "copy"
            assert np.array_equal(a.numpy().view(np.uint32), ref)
            assert np.array_equal(b.numpy().view(np.uint32), ref)
            m = zc.run(off, nb, check=True)     # the checker reads every entry: copied in bulk
            assert zc.last_mode == "copy" and zc.last_verdict.flags == 0
            assert oracle.check(g.offsets.numpy(), g.nbrs.numpy(), m.numpy().view(np.uint32)).flags == 0
        # pageable tensors fall back to the copy path
        g = graphs[0]
        zc.run(g.offsets.clone(), g.nbrs.clone(), serial=1)
        assert zc.last_mode == "copy"
    finally:
        zc.close()
        cp.close()


def test_host_session_on_a_side_stream(skp):
    """With stream= given, the session's copies run on that stream too: a busy
    current stream (a sleep kernel enqueued on it) must not let the pass read
    the previous graph's bytes out of the reused device buffers."""
    a, b = gg.rmat(11, 8, seed=1), gg.erdos_renyi(2048, 7000, seed=2)
    cp = skp.HostSession(max(a.n, b.n), max(a.nnz, b.nnz), zero_copy=False)
    side = torch.cuda.Stream()
    try:
        for g in (a, b, a):
            ref, _ = oracle.sgmm(g.offsets.numpy(), g.nbrs.numpy())
            torch.cuda._sleep(50_000_000)            # about 25 ms on the current stream
            m = cp.run(_pinned(g.offsets), _pinned(g.nbrs), stream=side, serial=1)
            assert cp.last_mode == "copy"
            assert np.array_equal(m.numpy().view(np.uint32), ref)
        torch.cuda.synchronize()
    finally:
        cp.close()


def _pageable_access():
    """cudaDevAttrPageableMemoryAccess: the device reads pageable host memory."""
    cudart = ctypes.CDLL("libcudart.so")
    v = ctypes.c_int(0)
    assert cudart.cudaDeviceGetAttribute(ctypes.byref(v), 88, torch.cuda.current_device()) == 0
    return v.value == 1


def test_pageable_memory_read_in_place_or_refused(skp):
    """The Python binding asks for pinned tensors; through the C ABI, pageable
    host memory is read in place where the device walks the host's page
    tables (Grace-Blackwell) and refused with MM_ERR_ARG elsewhere."""
    g = gg.rmat(11, 8, seed=9)
    with pytest.raises(ValueError):
        skp.Graph(g.offsets, g.nbrs, host_mapped=True)        # not pinned
    off, nb = g.offsets.clone(), g.nbrs.clone()                 # pageable host memory
    h = ctypes.c_void_p()
    rc = skp.lib.mm_create_csr(g.n, g.nnz, ctypes.c_void_p(off.data_ptr()),
                               ctypes.c_void_p(nb.data_ptr()), 2, None, ctypes.byref(h))
    if _pageable_access():
        assert rc == 0
        try:
            mate = torch.empty(g.n, dtype=torch.int32, device="cuda")
            o = skp.options(serial=1)
            assert skp.lib.mm_skipper(h, ctypes.byref(o), ctypes.c_void_p(mate.data_ptr()), None, 0,
                                      None, None) == 0
            ref, _ = oracle.sgmm(g.offsets.numpy(), g.nbrs.numpy())
            assert np.array_equal(_np(mate), ref)
        finally:
            skp.lib.mm_destroy(h)
    else:
        assert rc == 1 and b"cannot address" in skp.lib.mm_last_error()
    d = g.to("cuda")                                            # the context is still usable
    with skp.Graph(d.offsets, d.nbrs) as hg:
        assert hg.validate(hg.skipper()).flags == 0
