"""GPU parity: the CUDA path (through the C ABI) against the oracle.

Skipper's parallel result is any maximal matching (Section V-C: the output
varies between runs), so parallel runs are compared by the exact checker:
the oracle's verdict and the device checker's verdict must be identical field
by field, and both must say "valid maximal matching".  Where every maximal
matching is the same size (K_{a,b}, stars, K_n) or unique (disjoint edges),
the size or the bytes are compared too.  Serial mode walks rows and
neighbours in SGMM order and must reproduce SGMM byte for byte.
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
    return t.cpu().numpy().view(np.uint32) if t.dtype == torch.int32 else t.cpu().numpy()


def run(skp, csr, **kw):
    """Run through the C ABI; return (mate, pairs, oracle verdict, device verdict)."""
    off, nb = csr.offsets.numpy(), csr.nbrs.numpy()
    d = csr.to("cuda")
    with skp.Graph(d.offsets, d.nbrs) as h:
        mate, pairs, cnt = h.skipper(pairs=True, **kw)
        k = int(cnt.item())
        m = _np(mate)
        p = _np(pairs[:k]).reshape(-1, 2)
        vr = oracle.check(off, nb, m, p)
        vd = h.validate(mate, pairs[:k])
    return m, p, vr, vd


def assert_parity(vr, vd):
    assert vr.flags == 0, vr.as_dict()
    assert vd.as_dict() == vr.as_dict()


SMALL = {
    "fig1": lambda: gg.from_edges(4, torch.tensor([0, 0, 0, 1, 2]), torch.tensor([1, 2, 3, 2, 3])),
    "path101": lambda: gg.path(101),
    "star64": lambda: gg.star(64),
    "k3_17": lambda: gg.complete_bipartite(3, 17),
    "disjoint50": lambda: gg.disjoint_edges(50),
    "k9": lambda: gg.complete(9),
    "grid16x32": lambda: gg.grid(16, 32),
    "rmat10": lambda: gg.rmat(10, 16, seed=2),
    "er2k": lambda: gg.erdos_renyi(2000, 9000, seed=3),
}


@pytest.mark.parametrize("bits", [2, 8, 32])
@pytest.mark.parametrize("name", sorted(SMALL))
def test_serial_equals_sgmm(skp, name, bits):
    csr = SMALL[name]()
    ref_mate, ref_pairs = oracle.sgmm(csr.offsets.numpy(), csr.nbrs.numpy())
    m, p, vr, vd = run(skp, csr, status_bits=bits, serial=1)
    assert np.array_equal(m, ref_mate)
    assert np.array_equal(p, ref_pairs)   # ascending u = SGMM's push order on a symmetric CSR
    assert_parity(vr, vd)


@pytest.mark.parametrize("bits", [2, 8, 32])
@pytest.mark.parametrize("name", sorted(SMALL))
def test_parallel_valid_and_verdicts_identical(skp, name, bits):
    csr = SMALL[name]()
    _, ref_pairs = oracle.sgmm(csr.offsets.numpy(), csr.nbrs.numpy())
    for grain, id_loads in ((128, 1), (2048, 1), (128, 2), (2048, 2)):   # eager, selective
        m, p, vr, vd = run(skp, csr, status_bits=bits, grain=grain, id_loads=id_loads)
        assert_parity(vr, vd)
        assert 2 * len(p) >= len(ref_pairs)
        if name == "star64":
            assert len(p) == 1
        if name == "k3_17":
            assert len(p) == 3
        if name == "k9":
            assert len(p) == 4
        if name == "disjoint50":
            assert m.tolist() == [v ^ 1 for v in range(100)]


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_er_100k_1m(skp, bits):
    """Erdos-Renyi n=100,000, m=1,000,000 (2M directed entries)."""
    csr = gg.erdos_renyi(100_000, 1_000_000, seed=1)
    ref_mate, ref_pairs = oracle.sgmm(csr.offsets.numpy(), csr.nbrs.numpy())
    m, p, vr, vd = run(skp, csr, status_bits=bits, serial=1)
    assert np.array_equal(m, ref_mate)
    assert_parity(vr, vd)
    for grain, id_loads in ((256, 0), (2048, 0), (8192, 0), (2048, 2), (8192, 2)):
        m, p, vr, vd = run(skp, csr, status_bits=bits, grain=grain, id_loads=id_loads)
        assert_parity(vr, vd)
        assert 2 * len(p) >= len(ref_pairs)


@pytest.mark.parametrize("bits", [2, 8, 32])
@pytest.mark.parametrize("block", [32, 256, 512])
def test_launch_shapes(skp, bits, block):
    csr = gg.rmat(14, 16, seed=9)
    for bps, id_loads in ((0, 1), (1, 1), (0, 2)):
        m, p, vr, vd = run(skp, csr, status_bits=bits, block_threads=block, blocks_per_sm=bps,
                           id_loads=id_loads)
        assert_parity(vr, vd)


@pytest.mark.parametrize("bits", [2, 8, 32])
@pytest.mark.parametrize("symmetric", [0, 1])
def test_both_register_budgets_and_unit_orders(skp, bits, symmetric):
    """The plain and symmetric sweeps in their 40- and 32-register instances
    (blocks_per_sm 3 and 4 of 512 threads; 0 = the layout's default) and in
    both unit orders (ascending, dispersed runs; 0 = the layout's default), on
    a power-law graph, a grid and a graph whose units outnumber the warps
    several times over, all with the oracle's verdict."""
    for csr in (gg.rmat(14, 16, seed=12), gg.grid(200, 300), gg.erdos_renyi(300_000, 1_200_000, seed=13)):
        for bps in (0, 3, 4):
            for order in (0, 1, 2):
                m, p, vr, vd = run(skp, csr, status_bits=bits, block_threads=512, blocks_per_sm=bps,
                                   symmetric=symmetric, unit_order=order, grain=128)
                assert_parity(vr, vd)


def test_single_graph_autotuner(skp):
    """mm_autotune picks checked settings; the picked settings give the
    oracle's verdict on a power-law graph, a grid and an edge list."""
    for csr in (gg.rmat(14, 16, seed=14), gg.grid(300, 300)):
        off, nb = csr.offsets.numpy(), csr.nbrs.numpy()
        d = csr.to("cuda")
        with skp.Graph(d.offsets, d.nbrs) as h:
            o = h.autotune()
            assert o.status_bits in (2, 8, 32) and o.grain in (2048, 8192) and o.unit_order in (1, 2)
            mate = h.skipper(opts=o)
            vr = oracle.check(off, nb, _np(mate))
            assert vr.flags == 0 and h.validate(mate).as_dict() == vr.as_dict()
    csr = gg.rmat(12, 8, seed=15)
    src, dst = gg.edge_list(csr, "shuffle", seed=3)
    with skp.EdgeList(csr.n, src.cuda(), dst.cuda()) as h:
        o = h.autotune()
        mate = h.skipper(opts=o)
        vr = oracle.check_edges(csr.n, src.numpy(), dst.numpy(), _np(mate))
        assert vr.flags == 0 and h.validate(mate).as_dict() == vr.as_dict()


def test_unit_order_out_of_range_is_refused(skp):
    d = gg.grid(8, 8).to("cuda")
    with skp.Graph(d.offsets, d.nbrs) as h:
        with pytest.raises(skp.SkipperError) as e:
            h.skipper(unit_order=3)
        assert e.value.code == 1


def _manual(n, rows):
    off = [0]
    nb = []
    for r in rows:
        nb.extend(r)
        off.append(len(nb))
    assert len(off) == n + 1
    return gg.CSR(torch.tensor(off, dtype=torch.int64), torch.tensor(nb, dtype=torch.int32))


def test_loops_unsorted_rows_and_ragged_tail(skp):
    # self-loops, rows in arbitrary order, nnz = 13 (not a multiple of 4)
    csr = _manual(6, [[0, 3, 1], [0, 1, 2], [5, 1], [0, 3, 4], [3], [2]])
    ref_mate, _ = oracle.sgmm(csr.offsets.numpy(), csr.nbrs.numpy())
    for bits in (2, 8, 32):
        m, p, vr, vd = run(skp, csr, status_bits=bits, serial=1)
        assert np.array_equal(m, ref_mate)
        assert_parity(vr, vd)
        for grain in (128, 256):
            m, p, vr, vd = run(skp, csr, status_bits=bits, grain=grain)
            assert_parity(vr, vd)


def test_edges_stored_once(skp):
    """Non-symmetric CSR: each edge only in the row of its lower end (Section V-C)."""
    g = gg.rmat(12, 8, seed=4)
    off, nb = g.offsets.numpy(), g.nbrs.numpy()
    rows = np.repeat(np.arange(g.n), np.diff(off))
    keep = nb > rows
    cnt = np.bincount(rows[keep], minlength=g.n)
    off2 = np.zeros(g.n + 1, dtype=np.int64)
    off2[1:] = np.cumsum(cnt)
    csr = gg.CSR(torch.from_numpy(off2), torch.from_numpy(nb[keep].copy()))
    for bits in (2, 8, 32):
        m, p, vr, vd = run(skp, csr, status_bits=bits)
        assert_parity(vr, vd)
        ref_mate, _ = oracle.sgmm(off2, nb[keep])
        m, p, vr, vd = run(skp, csr, status_bits=bits, serial=1)
        assert np.array_equal(m, ref_mate)


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_symmetric_option(skp, bits):
    """symmetric=1: each edge tested once, from its lower endpoint's row; on a
    symmetric CSR the result is a maximal matching like any other (verdicts
    identical to the oracle's, sizes fixed where every maximal matching has
    one size); serial mode ignores the option."""
    for name in ("rmat10", "er2k", "grid16x32", "star64", "k3_17", "k9", "disjoint50", "path101"):
        csr = SMALL[name]()
        for grain, id_loads in ((128, 1), (2048, 1), (2048, 2)):
            m, p, vr, vd = run(skp, csr, status_bits=bits, grain=grain, symmetric=1, id_loads=id_loads)
            assert_parity(vr, vd)
            fixed = {"star64": 1, "k3_17": 3, "k9": 4, "disjoint50": 50}
            if name in fixed:
                assert len(p) == fixed[name]
        ref_mate, _ = oracle.sgmm(csr.offsets.numpy(), csr.nbrs.numpy())
        m, p, vr, vd = run(skp, csr, status_bits=bits, serial=1, symmetric=1)
        assert np.array_equal(m, ref_mate)
    for bits_ in (bits,):
        csr = gg.rmat(18, 16, seed=7)
        for id_loads in (1, 2):
            m, p, vr, vd = run(skp, csr, status_bits=bits_, grain=8192, symmetric=1, id_loads=id_loads)
            assert_parity(vr, vd)


def test_symmetric_option_is_the_callers_promise(skp):
    """On a CSR that holds each edge only in the row of its higher endpoint,
    symmetric=1 leaves every entry to a row that does not hold it: nothing is
    matched and the checker reports every entry uncovered."""
    n = 50
    csr = _manual(n, [[]] + [[i - 1] for i in range(1, n)])   # path, edge (i-1, i) in row i
    m, p, vr, vd = run(skp, csr, symmetric=1)
    assert m.tolist() == [NONE] * n and len(p) == 0
    assert vr.flags == oracle.V_UNCOVERED and vr.n_uncovered == n - 1
    assert vd.as_dict() == vr.as_dict()
    m, p, vr, vd = run(skp, csr)                                 # without the promise: maximal
    assert_parity(vr, vd)


def test_empty_rows_and_tiny_graphs(skp):
    # long runs of isolated vertices between short rows
    n = 3000
    u = torch.tensor([0, 1, 500, 501, 502, 2990, 2999, 1500], dtype=torch.int64)
    v = torch.tensor([1, 2, 501, 502, 503, 2999, 1500, 1000], dtype=torch.int64)
    csr = gg.from_edges(n, u, v)
    ref_mate, _ = oracle.sgmm(csr.offsets.numpy(), csr.nbrs.numpy())
    for bits in (2, 8, 32):
        m, p, vr, vd = run(skp, csr, status_bits=bits, serial=1)
        assert np.array_equal(m, ref_mate)
        for grain in (128, 2048):
            m, p, vr, vd = run(skp, csr, status_bits=bits, grain=grain)
            assert_parity(vr, vd)
    # no edges at all, and a single vertex
    for n in (1, 7):
        csr = gg.CSR(torch.zeros(n + 1, dtype=torch.int64), torch.zeros(0, dtype=torch.int32))
        m, p, vr, vd = run(skp, csr)
        assert m.tolist() == [NONE] * n and len(p) == 0
        assert_parity(vr, vd)


def test_misaligned_and_bad_graphs(skp):
    csr = gg.path(9).to("cuda")
    buf = torch.zeros(csr.nnz + 1, dtype=torch.int32, device="cuda")
    buf[1:] = csr.nbrs
    with pytest.raises(skp.SkipperError) as e:
        skp.Graph(csr.offsets, buf[1:])
    assert e.value.status == "MM_ERR_ARG"
    bad = csr.nbrs.clone()
    bad[3] = 9                       # id >= n
    with pytest.raises(skp.SkipperError) as e:
        skp.Graph(csr.offsets, bad)
    assert e.value.status == "MM_ERR_BAD_GRAPH"
    off = csr.offsets.clone()
    a, b = int(off[4]), int(off[5])
    off[4], off[5] = b, a            # not monotone
    with pytest.raises(skp.SkipperError) as e:
        skp.Graph(off, csr.nbrs)
    assert e.value.status == "MM_ERR_BAD_GRAPH"
    with pytest.raises(skp.SkipperError) as e:
        skp.Graph(csr.offsets, csr.nbrs).skipper(status_bits=16)
    assert e.value.status == "MM_ERR_ARG"


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_wait_limit_reports_timeout_and_context_survives(skp, bits):
    """A vertex left RESERVED by no thread: every wait on it runs out, the call
    returns MM_ERR_TIMEOUT (no trap, no hang), and the next call is normal."""
    csr = gg.rmat(12, 8, seed=6)
    d = csr.to("cuda")
    hub = int(torch.argmax(csr.offsets[1:] - csr.offsets[:-1]))
    with skp.Graph(d.offsets, d.nbrs) as h:
        for serial in (0, 1):
            with pytest.raises(skp.SkipperError) as e:
                h.skipper(status_bits=bits, serial=serial, poison_vertex=hub + 1, spin_limit=2000)
            assert e.value.status == "MM_ERR_TIMEOUT"
        mate = h.skipper(status_bits=bits)
        v = h.validate(mate)
        assert v.flags == 0


def test_validator_parity_on_corrupted_results(skp):
    csr = gg.erdos_renyi(3000, 12000, seed=8)
    off, nb = csr.offsets.numpy(), csr.nbrs.numpy()
    good, pairs = oracle.sgmm(off, nb)
    d = csr.to("cuda")
    rng = np.random.default_rng(0)
    cases = []
    m = good.copy(); a, b = pairs[5]; m[a] = m[b] = NONE; cases.append((m, None))      # uncovered
    m = good.copy(); m[pairs[7][0]] = NONE; cases.append((m, None))                    # asymmetric
    m = good.copy(); m[pairs[9][0]] = 2999 if pairs[9][0] != 2999 else 0; cases.append((m, None))
    m = good.copy(); m[11] = 1 << 30; cases.append((m, None))                          # out of range
    m = good.copy(); m[12] = 12; cases.append((m, None))                               # self
    m = good.copy(); unmatched = np.flatnonzero(m == NONE)
    if len(unmatched) >= 2:
        m[unmatched[0]], m[unmatched[1]] = unmatched[1], unmatched[0]                  # non-edge pair
    cases.append((m, None))
    cases.append((good, pairs[:-1]))                                                   # missing pair
    cases.append((good, np.vstack([pairs, pairs[:2]])))                                # repeats
    cases.append((good, pairs[:, ::-1].copy()))                                        # (high, low)
    cases.append((good, rng.permutation(pairs)))                                       # any order
    with skp.Graph(d.offsets, d.nbrs) as h:
        for m, p in cases:
            vr = oracle.check(off, nb, m, p)
            dm = torch.from_numpy(m.view(np.int32)).cuda()
            dp = None if p is None else torch.from_numpy(np.ascontiguousarray(p).astype(np.uint32).view(np.int32)).cuda()
            vd = h.validate(dm, dp)
            assert vd.as_dict() == vr.as_dict()
        assert sum(oracle.check(off, nb, m, p).flags != 0 for m, p in cases) == len(cases) - 1


def test_pairs_cap_nosync_and_timing(skp):
    csr = gg.rmat(13, 16, seed=12).to("cuda")
    with skp.Graph(csr.offsets, csr.nbrs) as h:
        mate, pairs, cnt = h.skipper(pairs=True, timing=1)
        t = h.timing()
        assert t["sweep_ms"] > 0 and t["units"] > 0
        k = int(cnt.item())
        mate2, pairs2, cnt2 = h.skipper(pairs=True, cap=5, serial=1)
        assert int(cnt2.item()) >= 5
        mate3, pairs3, cnt3 = h.skipper(pairs=True, serial=1)
        assert torch.equal(pairs2[:5], pairs3[:5])
        m = h.skipper(nosync=1)
        h.sync()
        assert h.validate(m).flags == 0
        # pairs list == {(u, mate[u]) : u < mate[u]} in ascending u
        mm = _np(mate).astype(np.int64)
        us = np.flatnonzero((mm != NONE) & (np.arange(len(mm)) < mm))
        assert np.array_equal(_np(pairs[:k]).reshape(-1, 2)[:, 0], us)


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_contention_shapes_and_rmat22(skp, bits):
    """RMAT scale 22 (ef 16), star with 1M leaves, path of 4M vertices,
    K_{2048,2048} and a 2048x2048 grid: verdicts identical to the oracle's."""
    shapes = {
        "rmat22": lambda: gg.rmat(22, 16, seed=1, device="cuda"),
        "star1m": lambda: gg.star(1_000_000, device="cuda"),
        "path4m": lambda: gg.path(4_000_000, device="cuda"),
        "k2048": lambda: gg.complete_bipartite(2048, 2048, device="cuda"),
        "grid2048": lambda: gg.grid(2048, 2048, device="cuda"),
    }
    for name, make in shapes.items():
        d = make()
        off, nb = d.offsets.cpu().numpy(), d.nbrs.cpu().numpy()
        _, ref_pairs = oracle.sgmm(off, nb)
        with skp.Graph(d.offsets, d.nbrs) as h:
            mate, pairs, cnt = h.skipper(status_bits=bits, pairs=True)
            k = int(cnt.item())
            vr = oracle.check(off, nb, _np(mate), _np(pairs[:k]).reshape(-1, 2))
            vd = h.validate(mate, pairs[:k])
        assert_parity(vr, vd)
        assert 2 * k >= len(ref_pairs), name
        if name == "star1m":
            assert k == 1
        if name == "k2048":
            assert k == 2048
        del d
        torch.cuda.empty_cache()


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_sweep_statistics(skp, bits):
    """stats=1 counts each successful claim once: matches == pairs in the result;
    every entry read at most once; conflicts fall in Table II's bins."""
    for csr in (gg.rmat(14, 16, seed=5), gg.complete_bipartite(64, 64), gg.star(5000)):
        d = csr.to("cuda")
        with skp.Graph(d.offsets, d.nbrs) as h:
            mate = h.skipper(status_bits=bits, stats=1)
            st = h.stats()
            v = h.validate(mate)
            assert v.flags == 0
            assert st["matches"] == v.n_pairs
            assert st["matches"] <= st["attempts"]
            assert 0 < st["entries_read"] <= csr.nnz
            assert st["conflicted_entries"] == sum(st["hist"])
            # every id read comes from a 128-bit load; the selective walk's loads
            # are a subset of the eager walk's
            assert 4 * st["id_loads"] >= st["entries_read"]
            assert 0 < st["id_loads_open"] <= st["id_loads"]
            assert st["conflicts"] >= st["conflicted_entries"]
            assert (st["max_conflicts"] > 0) == (st["conflicted_entries"] > 0)


def test_id_loads_option(skp):
    """id_loads: 0 (automatic), 1 (eager) and 2 (selective) give maximal
    matchings with oracle-identical verdicts on a ragged R-MAT; serial mode
    ignores it; any other value is refused before any device work."""
    csr = gg.rmat(16, 16, seed=11)
    for id_loads in (0, 1, 2):
        m, p, vr, vd = run(skp, csr, grain=2048, id_loads=id_loads)
        assert_parity(vr, vd)
    ref_mate, _ = oracle.sgmm(csr.offsets.numpy(), csr.nbrs.numpy())
    m, p, vr, vd = run(skp, csr, serial=1, id_loads=2)
    assert np.array_equal(m, ref_mate)
    d = csr.to("cuda")
    with skp.Graph(d.offsets, d.nbrs) as h:
        with pytest.raises(skp.SkipperError) as e:
            h.skipper(id_loads=3)
        assert e.value.status == "MM_ERR_ARG"


@pytest.mark.parametrize("bits", [2, 8])
def test_stage_windows_option(skp, bits):
    """stage_windows=1 (windows staged in shared memory by bulk copies one
    window ahead): maximal matchings with oracle-identical verdicts on ragged
    sizes, long runs of empty rows, one huge row and windows at the end of the
    arrays, with and without the symmetric filter; a CSR whose offsets are only
    8-byte aligned runs the unstaged walk; serial mode ignores the option."""
    graphs = [gg.rmat(14, 16, seed=21), gg.rmat(12, 4, seed=22), gg.star(5000), gg.grid(33, 47),
              gg.erdos_renyi(4099, 20000, seed=23), SMALL["path101"](), SMALL["fig1"]()]
    n = 3000
    rows = [[] for _ in range(n)]
    for x in range(0, n, 97):                       # short rows between long runs of empty rows
        for y in (x + 1, x + 45, x + 300):
            if y < n:
                rows[x].append(y)
                rows[y].append(x)
    graphs.append(_manual(n, [sorted(r) for r in rows]))
    for csr in graphs:
        for grain, sym in ((128, 0), (2048, 0), (8192, 0), (2048, 1)):
            m, p, vr, vd = run(skp, csr, status_bits=bits, grain=grain, symmetric=sym, stage_windows=1)
            assert_parity(vr, vd)
        ref_mate, _ = oracle.sgmm(csr.offsets.numpy(), csr.nbrs.numpy())
        m, p, vr, vd = run(skp, csr, status_bits=bits, serial=1, stage_windows=1)
        assert np.array_equal(m, ref_mate)
    # offsets 8-byte but not 16-byte aligned: the same call, unstaged
    csr = gg.rmat(13, 16, seed=24)
    big = torch.zeros(csr.n + 2, dtype=torch.int64, device="cuda")
    off = big[1:]
    off.copy_(csr.offsets.cuda())
    assert off.data_ptr() % 16 == 8
    nb = csr.nbrs.cuda()
    with skp.Graph(off, nb) as h:
        mate = h.skipper(status_bits=bits, stage_windows=1)
        vd = h.validate(mate)
    vr = oracle.check(csr.offsets.numpy(), csr.nbrs.numpy(), _np(mate))
    assert_parity(vr, vd)


def test_zero_vertex_graphs(skp):
    """n = 0 (offsets = [0], no entries) through every entry point: the pass,
    the pair list, the checker and the census on a CSR handle; an empty edge
    list; a multi-graph launch with an empty graph between two others; a
    request to the server; the host session; the allocation-free call."""
    import ctypes
    off = torch.zeros(1, dtype=torch.int64, device="cuda")
    nb = torch.zeros(0, dtype=torch.int32, device="cuda")
    for bits in (2, 8, 32):
        with skp.Graph(off, nb) as h:
            for kw in ({}, {"serial": 1}, {"symmetric": 1}, {"id_loads": 2}, {"stage_windows": 1}):
                mate, pairs, cnt = h.skipper(pairs=True, status_bits=bits, **kw)
                assert mate.numel() == 0 and int(cnt.item()) == 0
            v = h.validate(mate)
            assert v.flags == 0 and v.n_pairs == 0
            assert h.state_census() == {"acc": 0, "rsvd": 0, "mchd": 0, "other": 0}
        with skp.EdgeList(0, nb, nb) as h:
            assert h.skipper(status_bits=bits).numel() == 0
            assert h.skipper(status_bits=bits, serial=1).numel() == 0
            assert h.validate(torch.zeros(0, dtype=torch.int32, device="cuda")).flags == 0
    a, b = gg.path(9).to("cuda"), gg.star(20).to("cuda")
    mates = [torch.empty(9, dtype=torch.int32, device="cuda"), torch.empty(0, dtype=torch.int32, device="cuda"),
             torch.empty(21, dtype=torch.int32, device="cuda")]
    tri = [(a.offsets, a.nbrs, mates[0]), (off, nb, mates[1]), (b.offsets, b.nbrs, mates[2])]
    m = skp.Multi()
    try:
        m.run(tri)
        vs = m.validate(tri)
        assert [v.flags for v in vs] == [0, 0, 0] and vs[1].n_pairs == 0 and vs[2].n_pairs == 1
    finally:
        m.close()
    from paper_2507_04420_gb300.server import Server
    srv = Server(serial=True, status_bits=8)
    r = srv.submit(torch.zeros(1, dtype=torch.int64).pin_memory(), torch.zeros(0, dtype=torch.int32))
    assert r.wait(60) and r.error is None and r.verdict.flags == 0 and r.mate.numel() == 0
    srv.close()
    sess = skp.HostSession(4, 4)
    try:
        for zc in (True, False):
            sess.zero_copy = zc
            out = sess.run(torch.zeros(1, dtype=torch.int64).pin_memory(), torch.zeros(0, dtype=torch.int32))
            assert out.numel() == 0
    finally:
        sess.close()
    o = skp.options()
    rc = skp.lib.mm_skipper_static(0, 0, ctypes.c_void_p(off.data_ptr()), None, None, ctypes.byref(o), None)
    assert rc == 0, skp.lib.mm_last_error()
