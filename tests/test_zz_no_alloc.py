"""mm_skipper_static, the matching call that allocates no device memory.

Callers that cannot allocate device memory while they run -- a program whose
device memory all belongs to its own pool after start-up, a serving loop that
must not allocate per request, a plug-in living in a process whose allocator it
does not own -- use this call instead of mm_create_csr + mm_skipper.  Its
scratch sits in a fixed array inside the library.  These checks call it through
the C ABI twice in a row (the second call meets the first call's leftovers in
the shared array) and compare each result with the regular entry point's:

* serial mode is deterministic, so both calls must give the regular call's
  mate array byte for byte;
* the parallel pass may pick any maximal matching, so each result must pass
  the exact checker (device and oracle, identical verdicts) just as the
  regular call's result does, with at least half the pairs of SGMM.

This file is collected last so that a failure here cannot hide the others.
"""
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


def _static(skp, d, mate, **kw):
    o = skp.options(**kw)
    stream = ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    return skp.lib.mm_skipper_static(d.n, d.nnz, ctypes.c_void_p(d.offsets.data_ptr()),
                                     ctypes.c_void_p(d.nbrs.data_ptr()) if d.nnz else None,
                                     ctypes.c_void_p(mate.data_ptr()), ctypes.byref(o), stream)


def _np(t):
    return t.cpu().numpy().view(np.uint32)


GRAPHS = {
    "er_100k_1m": lambda: gg.erdos_renyi(100_000, 1_000_000, seed=1),
    "rmat16": lambda: gg.rmat(16, 16, seed=3),
    "grid512": lambda: gg.grid(512, 512),
    "star": lambda: gg.star(50_000),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_static_call_matches_regular_call(skp, name):
    csr = GRAPHS[name]()
    off, nb = csr.offsets.numpy(), csr.nbrs.numpy()
    d = csr.to("cuda")
    _, ref_pairs = oracle.sgmm(off, nb)
    with skp.Graph(d.offsets, d.nbrs) as h:
        regular_serial = _np(h.skipper(serial=1))
        regular = h.skipper()
        assert h.validate(regular).flags == 0
        for call in range(2):
            mate = torch.full((d.n,), 7, dtype=torch.int32, device="cuda")   # stale contents
            assert _static(skp, d, mate, serial=1) == 0, skp.lib.mm_last_error()
            assert np.array_equal(_np(mate), regular_serial), f"serial, call {call}"
        for call in range(2):
            mate = torch.full((d.n,), 7, dtype=torch.int32, device="cuda")
            assert _static(skp, d, mate) == 0, skp.lib.mm_last_error()
            vd = h.validate(mate)
            vr = oracle.check(off, nb, _np(mate))
            assert vr.flags == 0 and vd.as_dict() == vr.as_dict(), f"parallel, call {call}"
            assert 2 * vr.n_pairs >= len(ref_pairs)


def test_static_call_rejects_graphs_beyond_its_capacity(skp):
    limit = 7864064
    off = torch.zeros(limit + 2, dtype=torch.int64, device="cuda")   # limit + 1 vertices, no edges
    nb = torch.zeros(4, dtype=torch.int32, device="cuda")
    mate = torch.empty(limit + 1, dtype=torch.int32, device="cuda")
    o = skp.options()
    stream = ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    rc = skp.lib.mm_skipper_static(limit + 1, 0, ctypes.c_void_p(off.data_ptr()),
                                   ctypes.c_void_p(nb.data_ptr()), ctypes.c_void_p(mate.data_ptr()),
                                   ctypes.byref(o), stream)
    assert rc == 1 and b"capacity" in skp.lib.mm_last_error()
    # at the limit it runs
    rc = skp.lib.mm_skipper_static(limit, 0, ctypes.c_void_p(off.data_ptr()),
                                   ctypes.c_void_p(nb.data_ptr()), ctypes.c_void_p(mate.data_ptr()),
                                   ctypes.byref(o), stream)
    assert rc == 0
    assert bool((mate[:limit] == -1).all())


def test_static_call_refuses_what_it_cannot_run_and_says_why(skp):
    """Options that need a handle's own memory are refused, not ignored, and
    every refusal leaves its reason in mm_last_error()."""
    d = gg.grid(64, 64).to("cuda")
    mate = torch.empty(d.n, dtype=torch.int32, device="cuda")
    for kw in (dict(stats=1), dict(stage_windows=1), dict(symmetric=1), dict(id_loads=2),
               dict(timing=1), dict(status_bits=2)):
        assert _static(skp, d, mate, **kw) == 6, kw            # MM_ERR_UNSUPPORTED
        assert b"mm_skipper_static" in skp.lib.mm_last_error(), kw
    stream = ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    o = skp.options()
    rc = skp.lib.mm_skipper_static(d.n, d.nnz, ctypes.c_void_p(d.offsets.data_ptr()),
                                   ctypes.c_void_p(d.nbrs.data_ptr()), None, ctypes.byref(o), stream)
    assert rc == 1 and b"null mate" in skp.lib.mm_last_error()
    rc = skp.lib.mm_skipper_static(d.n, d.nnz, ctypes.c_void_p(d.offsets.data_ptr()),
                                   ctypes.c_void_p(d.nbrs.data_ptr() + 4), ctypes.c_void_p(mate.data_ptr()),
                                   ctypes.byref(o), stream)
    assert rc == 1 and b"16-byte aligned" in skp.lib.mm_last_error()
    # a refused call leaves the next one working
    assert _static(skp, d, mate) == 0, skp.lib.mm_last_error()
    assert h_valid(skp, d, mate)


def h_valid(skp, d, mate):
    with skp.Graph(d.offsets, d.nbrs) as h:
        return h.validate(mate).flags == 0
