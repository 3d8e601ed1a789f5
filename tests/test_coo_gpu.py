"""GPU parity for the edge-list input (Section V-C): mm_create_coo + mm_skipper
+ mm_validate through the C ABI against the edge-list oracle.

Serial mode takes the edges in list order and must equal SGMM over the list
byte for byte.  Parallel results are any maximal matching: the oracle's and
the device checker's verdicts must be identical field by field and say
"valid"; where every maximal matching has the same size (K_{a,b}, a star) or is
unique (disjoint edges), the size or the bytes are compared too.
"""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _lists():
    out = {}
    for name, make in {
        "rmat10": lambda: gg.rmat(10, 16, seed=2),
        "er2k": lambda: gg.erdos_renyi(2000, 9000, seed=3),
        "grid16x32": lambda: gg.grid(16, 32),
        "star300": lambda: gg.star(300),
        "k3_17": lambda: gg.complete_bipartite(3, 17),
        "path101": lambda: gg.path(101),
    }.items():
        g = make()
        for order in ("row", "shuffle"):
            s, d = gg.edge_list(g, order, seed=4)
            out[f"{name}_{order}"] = (g.n, s.numpy().view(np.uint32), d.numpy().view(np.uint32))
    return out


LISTS = _lists()


@pytest.mark.parametrize("bits", [2, 8, 32])
@pytest.mark.parametrize("name", sorted(LISTS))
def test_serial_equals_sgmm_over_the_list(skp, name, bits):
    n, src, dst = LISTS[name]
    ref, ref_pairs = oracle.sgmm_edges(n, src, dst)
    ds, dd = _dev(src), _dev(dst)
    with skp.EdgeList(n, ds, dd) as h:
        mate, pairs, cnt = h.skipper(pairs=True, serial=1, status_bits=bits)
        assert np.array_equal(_np(mate), ref)
        k = int(cnt.item())
        p = _np(pairs[:k]).reshape(-1, 2)
        assert np.array_equal(p, ref_pairs[np.argsort(ref_pairs[:, 0], kind="stable")])
        vd = h.validate(mate, pairs[:k])
        assert vd.as_dict() == oracle.check_edges(n, src, dst, ref, p).as_dict()


@pytest.mark.parametrize("bits", [2, 8, 32])
@pytest.mark.parametrize("grain", [128, 2048])
@pytest.mark.parametrize("name", sorted(LISTS))
def test_parallel_valid_and_verdicts_identical(skp, name, grain, bits):
    n, src, dst = LISTS[name]
    ds, dd = _dev(src), _dev(dst)
    with skp.EdgeList(n, ds, dd) as h:
        mate, pairs, cnt = h.skipper(pairs=True, status_bits=bits, grain=grain)
        k = int(cnt.item())
        m, p = _np(mate), _np(pairs[:k]).reshape(-1, 2)
        vr = oracle.check_edges(n, src, dst, m, p)
        vd = h.validate(mate, pairs[:k])
    assert vr.flags == 0, vr.as_dict()
    assert vd.as_dict() == vr.as_dict()
    if name.startswith("star"):
        assert k == 1
    if name.startswith("k3_17"):
        assert k == 3


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_unaligned_lists_ragged_tails_loops_and_repeats(skp, bits):
    """Lists that start off a 16-byte boundary take the 32-bit load path; the
    lengths leave a ragged last tile; loops and repeated edges are listed."""
    g = gg.rmat(11, 8, seed=9)
    s, d = gg.edge_list(g, "shuffle", seed=9)
    s, d = s.numpy().view(np.uint32), d.numpy().view(np.uint32)
    rng = np.random.default_rng(1)
    loops = rng.integers(0, g.n, 300).astype(np.uint32)
    rep = rng.integers(0, len(s), 500)
    src = np.concatenate([s, loops, d[rep]])
    dst = np.concatenate([d, loops, s[rep]])
    perm = rng.permutation(len(src))
    src, dst = src[perm], dst[perm]
    for off in (0, 1, 2, 3):
        m_len = len(src) - 37 - off
        bs, bd = _dev(src), _dev(dst)
        ds, dd = bs[off:off + m_len], bd[off:off + m_len]   # off 1..3: 4-byte aligned only
        hs, hd = src[off:off + m_len], dst[off:off + m_len]
        with skp.EdgeList(g.n, ds, dd) as h:
            mate = h.skipper(status_bits=bits, grain=256)
            vr = oracle.check_edges(g.n, hs, hd, _np(mate))
            assert vr.flags == 0 and h.validate(mate).as_dict() == vr.as_dict()
            ref, _ = oracle.sgmm_edges(g.n, hs, hd)
            assert np.array_equal(_np(h.skipper(status_bits=bits, serial=1)), ref)


def test_disjoint_edges_are_matched_exactly(skp):
    k = 5000
    a = np.arange(k, dtype=np.uint32)
    perm = np.random.default_rng(2).permutation(k)
    src, dst = (2 * a + 1)[perm], (2 * a)[perm]
    with skp.EdgeList(2 * k, _dev(src), _dev(dst)) as h:
        for bits in (2, 8, 32):
            m = _np(h.skipper(status_bits=bits))
            assert np.array_equal(m, np.arange(2 * k, dtype=np.uint32) ^ 1)


def test_empty_and_tiny_lists(skp):
    with skp.EdgeList(5, torch.zeros(0, dtype=torch.int32, device="cuda"),
                      torch.zeros(0, dtype=torch.int32, device="cuda")) as h:
        m = h.skipper()
        assert np.all(_np(m) == NONE)
        v = h.validate(m)
        assert v.flags == 0 and v.n_pairs == 0
    with skp.EdgeList(0, torch.zeros(0, dtype=torch.int32, device="cuda"),
                      torch.zeros(0, dtype=torch.int32, device="cuda")) as h:
        assert h.skipper().numel() == 0
    with skp.EdgeList(2, _dev([1]), _dev([0])) as h:
        assert _np(h.skipper()).tolist() == [1, 0]
    with skp.EdgeList(3, _dev([2, 1]), _dev([2, 1])) as h:   # loops only
        assert np.all(_np(h.skipper()) == NONE)


def test_bad_lists_are_rejected(skp):
    src, dst = _dev([0, 1, 7]), _dev([1, 2, 0])
    with pytest.raises(skp.SkipperError) as e:
        skp.EdgeList(4, src, dst)                      # id 7 >= n: checked at creation
    assert e.value.status == "MM_ERR_BAD_GRAPH"
    with skp.EdgeList(4, src, dst, check=False) as h:
        for serial in (0, 1):
            with pytest.raises(skp.SkipperError) as e:
                h.skipper(serial=serial)               # met during the pass
            assert e.value.status == "MM_ERR_BAD_GRAPH"
    with skp.EdgeList(3, _dev([0, 1]), _dev([1, 2])) as h:
        vb = torch.zeros(2, dtype=torch.int64, device="cuda")
        with pytest.raises(skp.SkipperError) as e:
            h.batched(vb, vb)
        assert e.value.status == "MM_ERR_UNSUPPORTED"
    with pytest.raises(ValueError):
        skp.EdgeList(3, _dev([0, 1]), _dev([1]))


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_wait_limit_reports_timeout_and_context_survives(skp, bits):
    g = gg.rmat(12, 8, seed=6)
    hub = int(torch.argmax(g.offsets[1:] - g.offsets[:-1]))
    s, d = gg.edge_list(g, "shuffle", seed=6)
    with skp.EdgeList(g.n, s.cuda(), d.cuda()) as h:
        for serial in (0, 1):
            with pytest.raises(skp.SkipperError) as e:
                h.skipper(status_bits=bits, serial=serial, poison_vertex=hub + 1, spin_limit=2000)
            assert e.value.status == "MM_ERR_TIMEOUT"
        assert h.validate(h.skipper(status_bits=bits)).flags == 0


def test_validator_parity_on_corrupted_results(skp):
    g = gg.erdos_renyi(3000, 12000, seed=8)
    s, d = gg.edge_list(g, "shuffle", seed=8)
    src, dst = s.numpy().view(np.uint32), d.numpy().view(np.uint32)
    good, pairs = oracle.sgmm_edges(g.n, src, dst)
    cases = []
    m = good.copy(); a, b = pairs[5]; m[a] = m[b] = NONE; cases.append((m, None))
    m = good.copy(); m[pairs[7][0]] = NONE; cases.append((m, None))
    m = good.copy(); m[11] = 1 << 30; cases.append((m, None))
    m = good.copy(); m[12] = 12; cases.append((m, None))
    m = good.copy(); un = np.flatnonzero(m == NONE)
    if len(un) >= 2:
        m[un[0]], m[un[1]] = un[1], un[0]
    cases.append((m, None))
    cases.append((good, pairs[:-1]))
    cases.append((good, np.vstack([pairs, pairs[:2]])))
    with skp.EdgeList(g.n, _dev(src), _dev(dst)) as h:
        for m, p in cases:
            vr = oracle.check_edges(g.n, src, dst, m, p)
            vd = h.validate(_dev(m), None if p is None else _dev(p))
            assert vd.as_dict() == vr.as_dict()
            assert vr.flags != 0


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_statistics(skp, bits):
    g = gg.rmat(14, 16, seed=5)
    s, d = gg.edge_list(g, "shuffle", seed=5)
    m_edges = s.numel()
    with skp.EdgeList(g.n, s.cuda(), d.cuda()) as h:
        mate = h.skipper(status_bits=bits, stats=1, grain=1024)
        st = h.stats()
        v = h.validate(mate)
    assert v.flags == 0
    assert st["entries_read"] == m_edges
    assert st["chunks"] == sum(-(-min(1024, m_edges - b) // 128) for b in range(0, m_edges, 1024))
    assert st["matches"] == v.n_pairs <= st["attempts"]
    assert st["conflicted_entries"] == sum(st["hist"])


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_rmat22_and_contention_shapes(skp, bits):
    """R-MAT 22 as raw generator draws (repeats and loops kept), a star with 1M
    leaves listed hub-first, K_{2048,2048} in row order."""
    shapes = {
        "rmat22_raw": lambda: (1 << 22, *gg.rmat_edges(22, 16 << 22, .57, .19, .19, 1, "cuda")),
        "star1m": lambda: (1_000_001, torch.zeros(1_000_000, dtype=torch.int32, device="cuda"),
                           torch.arange(1, 1_000_001, dtype=torch.int32, device="cuda")),
        "k2048": lambda: (4096, *gg.edge_list(gg.complete_bipartite(2048, 2048, device="cuda"), "row")),
    }
    for name, make in shapes.items():
        n, ds, dd = make()
        src, dst = _np(ds), _np(dd)
        with skp.EdgeList(n, ds.contiguous(), dd.contiguous()) as h:
            mate, pairs, cnt = h.skipper(status_bits=bits, pairs=True)
            k = int(cnt.item())
            vr = oracle.check_edges(n, src, dst, _np(mate), _np(pairs[:k]).reshape(-1, 2))
            vd = h.validate(mate, pairs[:k])
        assert vr.flags == 0 and vd.as_dict() == vr.as_dict(), name
        if name == "star1m":
            assert k == 1
        if name == "k2048":
            assert k == 2048
        del ds, dd
        torch.cuda.empty_cache()
