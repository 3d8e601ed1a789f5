"""Seeded synthetic graph generators producing symmetric CSR graphs.

This module is shared by the tests, the benchmark and the oracle-side
comparisons.  It holds none of the matching arithmetic: it only draws edges,
symmetrises them, sorts and de-duplicates each row.

Every graph is a pair ``(offsets int64[n+1], nbrs int32[nnz])``: row ``x``
lists the neighbours of ``x`` in ascending order, with no self-loops and no
duplicates, and the CSR is symmetric (``y`` in row ``x`` iff ``x`` in row
``y``).  Neighbour ids are non-negative and below 2**31, so the int32 storage
is read as uint32 by the matching library unchanged.

Randomness is counter-based: every draw is the splitmix64 output function
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) applied to a counter plus a seed-derived base, computed with
wrapping int64 tensor arithmetic.  The same seed therefore gives the same
graph on the CPU and on a CUDA device.

Shapes (stand-ins for the paper's workloads, Section VI-A / Table I):
  * ``rmat``   -- recursive-matrix (Kronecker-style) power-law graphs with
    per-bit quadrant choice (a, b, c, d), vertex ids randomly permuted; the
    synthetic g500 graph of Table I is of this family, and power-law social
    and web graphs are approximated by it.
  * ``erdos_renyi`` -- m distinct uniform random edges (low locality).
  * ``uniform`` -- m uniform random edge draws, de-duplicated.
  * closed-form shapes: ``path``, ``star``, ``complete_bipartite``,
    ``grid``, ``disjoint_edges``, ``complete``.
  * ``pack`` -- block-diagonal packing of several graphs with global ids
    and int64 per-graph vertex / entry base tables.
"""
from __future__ import annotations

import math
from typing import List, NamedTuple, Sequence

import torch

__all__ = [
    "CSR", "Packed", "mix64", "rmat", "erdos_renyi", "uniform", "path", "star",
    "complete_bipartite", "grid", "disjoint_edges", "complete", "from_edges", "pack",
    "batch_mix", "batch_packed", "unpack",
]

_MASK64 = (1 << 64) - 1


class CSR(NamedTuple):
    offsets: torch.Tensor  # int64 [n+1]
    nbrs: torch.Tensor     # int32 [nnz]

    @property
    def n(self) -> int:
        return int(self.offsets.numel()) - 1

    @property
    def nnz(self) -> int:
        return int(self.nbrs.numel())

    def to(self, device) -> "CSR":
        return CSR(self.offsets.to(device), self.nbrs.to(device))


class Packed(NamedTuple):
    csr: CSR               # union CSR with global ids
    vbase: torch.Tensor    # int64 [G+1]: graph g owns vertices [vbase[g], vbase[g+1])
    ebase: torch.Tensor    # int64 [G+1]: graph g owns entries  [ebase[g], ebase[g+1])


# ----------------------------------------------------------------------------
# counter-based randomness
# ----------------------------------------------------------------------------
def _s64(c: int) -> int:
    c &= _MASK64
    return c - (1 << 64) if c >= (1 << 63) else c


def _py_mix64(x: int) -> int:
    z = (x + 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def _lsr(z: torch.Tensor, k: int) -> torch.Tensor:
    return (z >> k) & ((1 << (64 - k)) - 1)


def mix64(x: torch.Tensor) -> torch.Tensor:
    """splitmix64 output function on an int64 tensor (wrapping arithmetic)."""
    z = x + _s64(0x9E3779B97F4A7C15)
    z = (z ^ _lsr(z, 30)) * _s64(0xBF58476D1CE4E5B9)
    z = (z ^ _lsr(z, 27)) * _s64(0x94D049BB133111EB)
    return z ^ _lsr(z, 31)


def _base(seed: int, stream: int) -> int:
    return _s64(_py_mix64(_py_mix64(seed & _MASK64) ^ (stream * 0x632BE59BD9B4E019)))


def _draw(seed: int, stream: int, start: int, count: int, device) -> torch.Tensor:
    """count 64-bit draws (int64) of stream `stream`, counters [start, start+count)."""
    ctr = torch.arange(start, start + count, dtype=torch.int64, device=device)
    return mix64(ctr + _base(seed, stream))


def _below(h: torch.Tensor, n: int) -> torch.Tensor:
    """Map 64-bit draws to [0, n) (63-bit modulo; bias below n / 2**63)."""
    return (h & 0x7FFFFFFFFFFFFFFF) % n


def _permutation(n: int, seed: int, device) -> torch.Tensor:
    """Seeded random permutation of [0, n): ranks of n distinct 64-bit draws."""
    h = _draw(seed, 7, 0, n, device)
    return torch.argsort(h, stable=True)


# ----------------------------------------------------------------------------
# CSR assembly
# ----------------------------------------------------------------------------
def _csr_from_directed(n: int, src: torch.Tensor, dst: torch.Tensor, chunks: int = 1) -> CSR:
    """Sort + de-duplicate directed entries (self-loops already removed) into CSR.

    `chunks` > 1 processes source-vertex ranges one at a time to bound the
    temporary memory of the sort on very large graphs."""
    device = src.device
    outs: List[torch.Tensor] = []
    deg = torch.zeros(n, dtype=torch.int64, device=device)
    step = max(1, -(-n // chunks))
    for lo in range(0, max(n, 1), step):
        hi = min(n, lo + step)
        if chunks == 1:
            s, d = src.to(torch.int64), dst.to(torch.int64)
        else:
            m = (src >= lo) & (src < hi)
            s, d = src[m].to(torch.int64), dst[m].to(torch.int64)
            del m
        key = torch.unique((s - lo) * n + d, sorted=True)
        del s, d
        rows = torch.div(key, n, rounding_mode="floor")
        deg[lo:hi] = torch.bincount(rows, minlength=hi - lo)
        outs.append((key - rows * n).to(torch.int32))
        del key, rows
    offsets = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(deg, 0, out=offsets[1:])
    nbrs = outs[0] if len(outs) == 1 else torch.cat(outs)
    return CSR(offsets, nbrs)


def from_edges(n: int, u: torch.Tensor, v: torch.Tensor, chunks: int = 1) -> CSR:
    """Symmetric CSR of the undirected edges {u_i, v_i}; loops and repeats dropped."""
    u = torch.as_tensor(u).to(torch.int64).reshape(-1)
    v = torch.as_tensor(v).to(torch.int64).reshape(-1).to(u.device)
    if u.numel() and (int(u.min()) < 0 or int(v.min()) < 0 or int(u.max()) >= n or int(v.max()) >= n):
        raise ValueError("edge endpoint outside [0, n)")
    keep = u != v
    u, v = u[keep], v[keep]
    if chunks == 1:
        return _csr_from_directed(n, torch.cat([u, v]), torch.cat([v, u]))
    # large graphs: keep the two directions apart until each source range is cut out
    return _csr_from_directed_pairs(n, u, v, chunks)


def _csr_from_directed_pairs(n: int, u: torch.Tensor, v: torch.Tensor, chunks: int) -> CSR:
    device = u.device
    outs: List[torch.Tensor] = []
    deg = torch.zeros(n, dtype=torch.int64, device=device)
    step = max(1, -(-n // chunks))
    for lo in range(0, max(n, 1), step):
        hi = min(n, lo + step)
        m1 = (u >= lo) & (u < hi)
        m2 = (v >= lo) & (v < hi)
        s = torch.cat([u[m1], v[m2]]).to(torch.int64)
        d = torch.cat([v[m1], u[m2]]).to(torch.int64)
        del m1, m2
        key = torch.unique((s - lo) * n + d, sorted=True)
        del s, d
        rows = torch.div(key, n, rounding_mode="floor")
        deg[lo:hi] = torch.bincount(rows, minlength=hi - lo)
        outs.append((key - rows * n).to(torch.int32))
        del key, rows
    offsets = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(deg, 0, out=offsets[1:])
    return CSR(offsets, torch.cat(outs) if len(outs) > 1 else outs[0])


# ----------------------------------------------------------------------------
# random families
# ----------------------------------------------------------------------------
def rmat_edges(scale: int, m: int, a: float, b: float, c: float, seed: int,
               device="cpu", permute: bool = True, chunk: int = 1 << 25):
    """m R-MAT edge draws on 2**scale vertices (int32 endpoint tensors).

    Each edge picks one quadrant per bit level: (0,0) with probability a,
    (0,1) with b, (1,0) with c and (1,1) with d = 1 - a - b - c, using 32-bit
    uniform draws compared with integer thresholds (exact on every device)."""
    if not (0 < scale <= 31):
        raise ValueError("scale must be in 1..31")
    ta = int(a * 2**32)
    tb = int((a + b) * 2**32)
    tc = int((a + b + c) * 2**32)
    per_edge = (scale + 1) // 2
    us, vs = [], []
    for start in range(0, m, chunk):
        cnt = min(chunk, m - start)
        u = torch.zeros(cnt, dtype=torch.int64, device=device)
        v = torch.zeros(cnt, dtype=torch.int64, device=device)
        ctr = torch.arange(start, start + cnt, dtype=torch.int64, device=device) * per_edge
        h = None
        for lvl in range(scale):
            if lvl % 2 == 0:
                h = mix64(ctr + (lvl // 2) + _base(seed, 1))
                r = h & 0xFFFFFFFF
            else:
                r = _lsr(h, 32)
            bu = r >= tb
            bv = ((r >= ta) & (r < tb)) | (r >= tc)
            u = (u << 1) | bu.to(torch.int64)
            v = (v << 1) | bv.to(torch.int64)
        us.append(u.to(torch.int32))
        vs.append(v.to(torch.int32))
        del u, v, ctr, h
    u = torch.cat(us) if len(us) > 1 else us[0]
    v = torch.cat(vs) if len(vs) > 1 else vs[0]
    del us, vs
    if permute:
        p = _permutation(1 << scale, seed, device).to(torch.int32)
        u = p[u.long()]
        v = p[v.long()]
    return u, v


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, device="cpu", permute: bool = True, chunks: int = 1) -> CSR:
    """R-MAT graph: 2**scale vertices, edge_factor * 2**scale edge draws, symmetrised,
    loops and duplicates dropped (so nnz <= 2 * edge_factor * 2**scale)."""
    n = 1 << scale
    u, v = rmat_edges(scale, edge_factor * n, a, b, c, seed, device, permute)
    keep = u != v
    u, v = u[keep], v[keep]
    del keep
    if chunks == 1:
        u64, v64 = u.to(torch.int64), v.to(torch.int64)
        del u, v
        return _csr_from_directed(n, torch.cat([u64, v64]), torch.cat([v64, u64]))
    return _csr_from_directed_pairs(n, u, v, chunks)


def uniform(n: int, m: int, seed: int = 1, device="cpu", chunks: int = 1) -> CSR:
    """m uniform random endpoint pairs on n vertices; loops and repeats dropped."""
    u = torch.empty(m, dtype=torch.int32, device=device)
    v = torch.empty(m, dtype=torch.int32, device=device)
    step = 1 << 25
    for s in range(0, m, step):
        k = min(step, m - s)
        u[s:s + k] = _below(_draw(seed, 2, s, k, device), n).to(torch.int32)
        v[s:s + k] = _below(_draw(seed, 3, s, k, device), n).to(torch.int32)
    keep = u != v
    u, v = u[keep], v[keep]
    if chunks == 1:
        u64, v64 = u.to(torch.int64), v.to(torch.int64)
        return _csr_from_directed(n, torch.cat([u64, v64]), torch.cat([v64, u64]))
    return _csr_from_directed_pairs(n, u, v, chunks)


def erdos_renyi(n: int, m: int, seed: int = 1, device="cpu") -> CSR:
    """Exactly m distinct undirected edges drawn uniformly (no loops, no repeats).

    Candidates are drawn until at least m distinct pairs exist; the m kept are
    those with the smallest seeded 64-bit keys, a uniform random subset."""
    if m > n * (n - 1) // 2:
        raise ValueError("m exceeds n(n-1)/2")
    keys = torch.empty(0, dtype=torch.int64, device=device)
    drawn = 0
    while keys.numel() < m:
        k = max(1024, int((m - keys.numel()) * 1.15) + 64)
        u = _below(_draw(seed, 4, drawn, k, device), n)
        v = _below(_draw(seed, 5, drawn, k, device), n)
        drawn += k
        keep = u != v
        lo = torch.minimum(u, v)[keep]
        hi = torch.maximum(u, v)[keep]
        keys = torch.unique(torch.cat([keys, lo * n + hi]))
    order = torch.argsort(mix64(keys + _base(seed, 6)), stable=True)[:m]
    keys = keys[order]
    lo = torch.div(keys, n, rounding_mode="floor")
    hi = keys - lo * n
    return _csr_from_directed(n, torch.cat([lo, hi]), torch.cat([hi, lo]))


# ----------------------------------------------------------------------------
# closed-form shapes (natural ids)
# ----------------------------------------------------------------------------
def path(n: int, device="cpu") -> CSR:
    """Path 0-1-2-...-(n-1)."""
    i = torch.arange(max(n - 1, 0), dtype=torch.int64, device=device)
    return from_edges(n, i, i + 1)


def star(k: int, device="cpu") -> CSR:
    """Centre 0 with leaves 1..k."""
    leaves = torch.arange(1, k + 1, dtype=torch.int64, device=device)
    return from_edges(k + 1, torch.zeros_like(leaves), leaves)


def complete_bipartite(a: int, b: int, device="cpu") -> CSR:
    """K_{a,b}: left 0..a-1, right a..a+b-1."""
    left = torch.arange(a, dtype=torch.int64, device=device).repeat_interleave(b)
    right = a + torch.arange(b, dtype=torch.int64, device=device).repeat(a)
    return from_edges(a + b, left, right)


def grid(rows: int, cols: int, device="cpu") -> CSR:
    """rows x cols 4-neighbour grid, row-major ids r*cols + c."""
    r = torch.arange(rows, dtype=torch.int64, device=device)
    c = torch.arange(cols, dtype=torch.int64, device=device)
    rr, cc = torch.meshgrid(r, c, indexing="ij")
    ids = rr * cols + cc
    hu, hv = ids[:, :-1].reshape(-1), ids[:, 1:].reshape(-1)
    vu, vv = ids[:-1, :].reshape(-1), ids[1:, :].reshape(-1)
    return from_edges(rows * cols, torch.cat([hu, vu]), torch.cat([hv, vv]))


def disjoint_edges(k: int, device="cpu") -> CSR:
    """k disjoint edges (2i, 2i+1)."""
    i = torch.arange(k, dtype=torch.int64, device=device)
    return from_edges(2 * k, 2 * i, 2 * i + 1)


def complete(n: int, device="cpu") -> CSR:
    """K_n."""
    iu = torch.triu_indices(n, n, offset=1, device=device)
    return from_edges(n, iu[0], iu[1])


# ----------------------------------------------------------------------------
# batches
# ----------------------------------------------------------------------------
def edge_list(g: CSR, order: str = "row", seed: int = 1):
    """Each undirected edge of a symmetric CSR listed once, as (src, dst) int32 tensors.

    order="row": CSR row order with src < dst (a sorted coordinate list).
    order="shuffle": the same edges in a seeded random order, each one's
    direction flipped by a seeded coin (a list in no particular order)."""
    dev = g.offsets.device
    deg = g.offsets[1:] - g.offsets[:-1]
    rows = torch.repeat_interleave(torch.arange(g.n, dtype=torch.int32, device=dev), deg)
    keep = rows < g.nbrs
    src, dst = rows[keep], g.nbrs[keep]
    del rows, keep
    if order == "row":
        return src, dst
    if order != "shuffle":
        raise ValueError("order must be 'row' or 'shuffle'")
    m = src.numel()
    perm = torch.argsort(_draw(seed, 11, 0, m, dev), stable=True)
    src, dst = src[perm], dst[perm]
    del perm
    flip = (_draw(seed, 12, 0, m, dev) & 1).bool()
    return torch.where(flip, dst, src), torch.where(flip, src, dst)


def pack(graphs: Sequence[CSR], device=None, local: bool = False) -> Packed:
    """Block-diagonal packing: graph g's vertex x becomes vbase[g] + x (with
    local=True the neighbour ids stay local to each graph; only the offsets
    become batch entry indices)."""
    if device is None:
        device = graphs[0].offsets.device if graphs else "cpu"
    ns = [g.n for g in graphs]
    es = [g.nnz for g in graphs]
    vbase = torch.zeros(len(graphs) + 1, dtype=torch.int64)
    ebase = torch.zeros(len(graphs) + 1, dtype=torch.int64)
    if graphs:
        vbase[1:] = torch.cumsum(torch.tensor(ns, dtype=torch.int64), 0)
        ebase[1:] = torch.cumsum(torch.tensor(es, dtype=torch.int64), 0)
    if int(vbase[-1]) >= 2**31 and not local:
        raise ValueError("packed vertex count must stay below 2**31")
    offs = [torch.zeros(1, dtype=torch.int64, device=device)]
    nb = []
    for g, gr in enumerate(graphs):
        offs.append(gr.offsets[1:].to(device) + int(ebase[g]))
        nb.append(gr.nbrs.to(device) + (0 if local else int(vbase[g])))
    offsets = torch.cat(offs)
    nbrs = torch.cat(nb) if nb else torch.zeros(0, dtype=torch.int32, device=device)
    return Packed(CSR(offsets, nbrs.to(torch.int32)), vbase.to(device), ebase.to(device))


def batch_mix(num_graphs: int, m_lo: float, m_hi: float, seed: int = 1, device="cpu",
              kinds=("er", "rmat", "grid")) -> List[CSR]:
    """num_graphs graphs with edge counts log-uniform in [m_lo, m_hi], cycling through
    ER, R-MAT (edge factor uniform in 8..32, n = 2**round(log2(m / ef))) and 2-D grids
    (side round(sqrt(m / 2)))."""
    h = _draw(seed, 8, 0, 3 * num_graphs, "cpu")
    uni = (_lsr(h, 11).to(torch.float64) / float(1 << 53)).tolist()
    out: List[CSR] = []
    for g in range(num_graphs):
        m = int(round(math.exp(math.log(m_lo) + uni[3 * g] * (math.log(m_hi) - math.log(m_lo)))))
        kind = kinds[g % len(kinds)]
        ef = 8 + int(uni[3 * g + 1] * 25) % 25
        gseed = seed * 1000003 + g
        if kind == "er":
            n = max(16, int(round(2 * m / ef)))
            out.append(erdos_renyi(n, min(m, n * (n - 1) // 2), gseed, device))
        elif kind == "rmat":
            scale = max(4, int(round(math.log2(max(m / ef, 16)))))
            n = 1 << scale
            u, v = rmat_edges(scale, m, 0.57, 0.19, 0.19, gseed, device)
            out.append(from_edges(n, u, v))
        else:
            side = max(2, int(round(math.sqrt(m / 2))))
            out.append(grid(side, side, device))
    return out


def unpack(packed: Packed, g: int) -> CSR:
    """Graph g of a block-diagonal packing as a standalone CSR with local ids."""
    v0, v1 = int(packed.vbase[g]), int(packed.vbase[g + 1])
    e0, e1 = int(packed.ebase[g]), int(packed.ebase[g + 1])
    off = packed.csr.offsets[v0:v1 + 1] - e0
    nb = packed.csr.nbrs[e0:e1] - v0
    return CSR(off.contiguous(), nb.contiguous())


def _scramble(x: torch.Tensor, bits: torch.Tensor, a1: torch.Tensor, a2: torch.Tensor) -> torch.Tensor:
    """A bijection of [0, 2**bits) per element: odd multiply, xor-shift, odd multiply (mod 2**bits)."""
    mask = (torch.ones_like(bits) << bits) - 1
    x = (x * a1) & mask
    x = x ^ (x >> ((bits + 1) // 2))
    return (x * a2) & mask


def batch_packed(num_graphs: int, m_lo: float, m_hi: float, seed: int = 1, device="cpu",
                 chunks: int = 1, kinds=("er", "rmat", "grid")):
    """A packed batch of num_graphs graphs drawn in one vectorised pass.

    Edge counts are log-uniform in [m_lo, m_hi]; graph g is kinds[g % len(kinds)]:
    ER (n = 2m/ef, m uniform endpoint draws), R-MAT (edge factor ef uniform in 8..32,
    n = 2**round(log2(m/ef)), a/b/c/d = .57/.19/.19/.05, ids scrambled by a per-graph
    bijection) or a side x side grid (side = round(sqrt(m/2))).  Loops and repeats are
    dropped.  Returns (Packed, kinds list)."""
    G = num_graphs
    h = _draw(seed, 8, 0, 3 * G, "cpu")
    uni = (_lsr(h, 11).to(torch.float64) / float(1 << 53)).tolist()
    ms, ns, kind_of, efs, scales, sides = [], [], [], [], [], []
    for g in range(G):
        m = int(round(math.exp(math.log(m_lo) + uni[3 * g] * (math.log(m_hi) - math.log(m_lo)))))
        k = kinds[g % len(kinds)]
        ef = 8 + int(uni[3 * g + 1] * 25) % 25
        sc = side = 0
        if k == "er":
            n = max(16, int(round(2 * m / ef)))
        elif k == "rmat":
            sc = max(4, int(round(math.log2(max(m / ef, 16)))))
            n = 1 << sc
        else:
            side = max(2, int(round(math.sqrt(m / 2))))
            n = side * side
        ms.append(m); ns.append(n); kind_of.append(k); efs.append(ef); scales.append(sc); sides.append(side)
    vbase = torch.zeros(G + 1, dtype=torch.int64)
    vbase[1:] = torch.cumsum(torch.tensor(ns, dtype=torch.int64), 0)
    N = int(vbase[-1])
    if N >= 2**31:
        raise ValueError("packed vertex count must stay below 2**31")
    vb = vbase.to(device)
    us, vs = [], []

    def per_edge(ids, counts):
        return torch.repeat_interleave(torch.tensor(ids, dtype=torch.int64, device=device),
                                       torch.tensor(counts, dtype=torch.int64, device=device))

    # Erdos-Renyi members
    er = [g for g in range(G) if kind_of[g] == "er"]
    if er:
        ge = per_edge(er, [ms[g] for g in er])
        nn = torch.tensor(ns, dtype=torch.int64, device=device)[ge]
        cnt = ge.numel()
        u = (_draw(seed, 20, 0, cnt, device) & 0x7FFFFFFFFFFFFFFF) % nn
        v = (_draw(seed, 21, 0, cnt, device) & 0x7FFFFFFFFFFFFFFF) % nn
        us.append(u + vb[ge]); vs.append(v + vb[ge])
    # R-MAT members
    rm = [g for g in range(G) if kind_of[g] == "rmat"]
    if rm:
        ge = per_edge(rm, [ms[g] for g in rm])
        cnt = ge.numel()
        sc_all = torch.tensor(scales, dtype=torch.int64, device=device)
        s_e = sc_all[ge]
        smax = int(max(scales[g] for g in rm))
        u = torch.zeros(cnt, dtype=torch.int64, device=device)
        v = torch.zeros(cnt, dtype=torch.int64, device=device)
        ta, tb, tc = int(0.57 * 2**32), int(0.76 * 2**32), int(0.95 * 2**32)
        per = (smax + 1) // 2
        ctr = torch.arange(cnt, dtype=torch.int64, device=device) * per
        hh = None
        for lvl in range(smax):
            if lvl % 2 == 0:
                hh = mix64(ctr + lvl // 2 + _base(seed, 22))
                r = hh & 0xFFFFFFFF
            else:
                r = _lsr(hh, 32)
            u = (u << 1) | (r >= tb).to(torch.int64)
            v = (v << 1) | (((r >= ta) & (r < tb)) | (r >= tc)).to(torch.int64)
        u = u >> (smax - s_e)
        v = v >> (smax - s_e)
        gconst = torch.tensor([_py_mix64(seed * 7919 + g) & 0xFFFFFFFF for g in range(G)],
                              dtype=torch.int64, device=device)
        a1 = (gconst[ge] << 1) | 1
        a2 = ((gconst[ge] >> 7) << 1) | 1
        u = _scramble(u, s_e, a1, a2)
        v = _scramble(v, s_e, a1, a2)
        us.append(u + vb[ge]); vs.append(v + vb[ge])
    # grid members
    gr = [g for g in range(G) if kind_of[g] == "grid"]
    if gr:
        for horiz in (True, False):
            cnts = [sides[g] * (sides[g] - 1) for g in gr]
            ge = per_edge(gr, cnts)
            side = torch.tensor(sides, dtype=torch.int64, device=device)[ge]
            first = torch.zeros(len(gr) + 1, dtype=torch.int64)
            first[1:] = torch.cumsum(torch.tensor(cnts, dtype=torch.int64), 0)
            local = torch.arange(ge.numel(), dtype=torch.int64, device=device) - \
                first.to(device)[:-1].repeat_interleave(torch.tensor(cnts, device=device))
            if horiz:   # (r, c) - (r, c+1)
                r, c = local // (side - 1), local % (side - 1)
                a = r * side + c
                b = a + 1
            else:       # (r, c) - (r+1, c)
                r, c = local // side, local % side
                a = r * side + c
                b = a + side
            us.append(a + vb[ge]); vs.append(b + vb[ge])
    u = torch.cat(us)
    v = torch.cat(vs)
    keep = u != v
    u, v = u[keep].to(torch.int32), v[keep].to(torch.int32)
    csr = _csr_from_directed_pairs(N, u, v, max(1, chunks))
    ebase = csr.offsets[vb]
    return Packed(csr, vb, ebase), kind_of
