"""Oracle for Skipper's maximal matching -- TEST INFRASTRUCTURE ONLY.

Plain, single-thread C (``sgmm.c``, ``check.c``) compiled with gcc and called
through ctypes:

* ``sgmm``  -- Sequential Greedy Maximal Matching (Section II-B; the
  sequential algorithm the paper measures Skipper against, Figs. 9-11).
* ``check`` -- the exact maximal-matching checker (Section II-B's rule: every
  edge touches an output edge, no two output edges share an endpoint).
* ``cpu_skipper`` (``skipper_cpu.c``) -- not an oracle: Algorithm 1 on host
  threads, the paper's own setting, a CPU baseline for the benchmark
  (parallelization gain and serial slowdown, Section VI-D); its results are
  checked with ``check``.
* ``sgmm_edges`` / ``check_edges`` (``edges.c``) -- the same two over a list
  of edges in coordinate form (Section V-C: Skipper reads such a list
  directly), SGMM taking the edges in list order.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA library under
``paper_2507_04420_gb300/`` and never imports it.

Parity pins live in ``tests/test_oracle.py``: the worked example of Fig. 1
(``tests/golden/fig1_worked_example.txt``), closed forms (path, star,
K_{a,b}, disjoint edges, K_n, grid), and brute force over every graph on up to
six vertices.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = [os.path.join(_HERE, "sgmm.c"), os.path.join(_HERE, "check.c"),
            os.path.join(_HERE, "edges.c"), os.path.join(_HERE, "skipper_cpu.c")]
_lock = threading.Lock()
_lib = None

NONE = 0xFFFFFFFF

V_RANGE, V_ASYM, V_NONEDGE, V_UNCOVERED, V_PAIRS = 1, 2, 4, 8, 16


class Verdict(ctypes.Structure):
    _fields_ = [
        ("flags", ctypes.c_uint32),
        ("pad", ctypes.c_uint32),
        ("n_matched", ctypes.c_uint64),
        ("n_pairs", ctypes.c_uint64),
        ("n_bad_range", ctypes.c_uint64),
        ("n_asym", ctypes.c_uint64),
        ("n_nonedge", ctypes.c_uint64),
        ("n_uncovered", ctypes.c_uint64),
        ("n_pairs_bad", ctypes.c_uint64),
        ("first_bad_vertex", ctypes.c_uint64),
        ("first_uncovered", ctypes.c_uint64),
    ]

    FIELDS = ("flags", "n_matched", "n_pairs", "n_bad_range", "n_asym", "n_nonedge",
              "n_uncovered", "n_pairs_bad", "first_bad_vertex", "first_uncovered")

    def as_dict(self):
        return {k: int(getattr(self, k)) for k in self.FIELDS}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no target-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SOURCES)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-pthread",
                               "-shared", "-fPIC", "-o", tmp, *_SOURCES])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i64, p = ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p
            lib.oracle_sgmm.argtypes = [u64, p, p, p, p]
            lib.oracle_sgmm.restype = i64
            lib.oracle_sgmm_timed.argtypes = [u64, p, p, p, ctypes.POINTER(ctypes.c_double)]
            lib.oracle_sgmm_timed.restype = i64
            lib.oracle_sgmm_rows_timed.argtypes = [u64, p, p, u64, u64, p,
                                                   ctypes.POINTER(ctypes.c_double)]
            lib.oracle_sgmm_rows_timed.restype = i64
            lib.oracle_check.argtypes = [u64, p, p, p, p, u64, ctypes.POINTER(Verdict)]
            lib.oracle_check.restype = ctypes.c_int
            lib.cpu_skipper.argtypes = [u64, p, p, u64, u64, ctypes.c_int, u64, ctypes.c_int, p,
                                        ctypes.POINTER(ctypes.c_double)]
            lib.cpu_skipper.restype = i64
            lib.oracle_sgmm_edges.argtypes = [u64, u64, p, p, p, p]
            lib.oracle_sgmm_edges.restype = i64
            lib.oracle_check_edges.argtypes = [u64, u64, p, p, p, p, u64, ctypes.POINTER(Verdict)]
            lib.oracle_check_edges.restype = ctypes.c_int
            _lib = lib
    return _lib


def _u32(a):
    a = np.ascontiguousarray(np.asarray(a))
    return a.view(np.uint32) if a.dtype == np.int32 else a.astype(np.uint32, copy=False)


def _csr(offsets, nbrs):
    offsets = np.ascontiguousarray(np.asarray(offsets), dtype=np.int64)
    nbrs = _u32(nbrs)
    if offsets.ndim != 1 or offsets.size < 1:
        raise ValueError("offsets must be a 1-D array of n+1 entries")
    n = offsets.size - 1
    if offsets[0] != 0 or offsets[-1] != nbrs.size or np.any(np.diff(offsets) < 0):
        raise ValueError("offsets must start at 0, be non-decreasing and end at len(nbrs)")
    return n, offsets, nbrs


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def sgmm(offsets, nbrs):
    """SGMM over the CSR: returns (mate uint32[n], pairs uint32[k, 2])."""
    n, offsets, nbrs = _csr(offsets, nbrs)
    mate = np.empty(n, dtype=np.uint32)
    pairs = np.empty((max(n // 2, 1), 2), dtype=np.uint32)
    k = _load().oracle_sgmm(n, _ptr(offsets), _ptr(nbrs), _ptr(mate), _ptr(pairs))
    if k < 0:
        raise ValueError("oracle_sgmm failed (neighbour id out of range or no memory)")
    return mate, pairs[:k].copy()


def sgmm_timed(offsets, nbrs):
    """SGMM with its edge walk timed in C; returns (mate, seconds)."""
    n, offsets, nbrs = _csr(offsets, nbrs)
    mate = np.empty(n, dtype=np.uint32)
    sec = ctypes.c_double(0.0)
    k = _load().oracle_sgmm_timed(n, _ptr(offsets), _ptr(nbrs), _ptr(mate), ctypes.byref(sec))
    if k < 0:
        raise ValueError("oracle_sgmm failed")
    return mate, float(sec.value)


def sgmm_rows_timed(offsets, nbrs, row_end):
    """SGMM over rows [0, row_end) only (a bounded sample of a large graph).

    Returns (pairs taken, seconds, CSR entries in the sampled rows)."""
    offsets = np.ascontiguousarray(np.asarray(offsets), dtype=np.int64)
    nbrs = _u32(nbrs)
    n = offsets.size - 1
    row_end = int(min(row_end, n))
    mate = np.full(n, NONE, dtype=np.uint32)
    sec = ctypes.c_double(0.0)
    k = _load().oracle_sgmm_rows_timed(n, _ptr(offsets), _ptr(nbrs), 0, row_end, _ptr(mate),
                                       ctypes.byref(sec))
    if k < 0:
        raise ValueError("oracle_sgmm_rows_timed failed")
    return int(k), float(sec.value), int(offsets[row_end])


def check(offsets, nbrs, mate, pairs=None) -> Verdict:
    """Exact checker; returns a Verdict (flags == 0 means a valid maximal matching)."""
    n, offsets, nbrs = _csr(offsets, nbrs)
    mate = _u32(mate)
    if mate.size != n:
        raise ValueError("mate must have n entries")
    count = 0
    pp = None
    if pairs is not None:
        pairs = _u32(pairs).reshape(-1, 2)
        count = pairs.shape[0]
        if count == 0:
            pairs = np.zeros((1, 2), dtype=np.uint32)   # a valid pointer; nothing is read
        pp = _ptr(pairs)
    v = Verdict()
    rc = _load().oracle_check(n, _ptr(offsets), _ptr(nbrs), _ptr(mate), pp, count, ctypes.byref(v))
    if rc != 0:
        raise MemoryError("oracle_check: no memory")
    return v


def _edges(n, src, dst):
    src, dst = _u32(src), _u32(dst)
    if src.ndim != 1 or src.shape != dst.shape:
        raise ValueError("src and dst must be 1-D arrays of the same length")
    return int(n), src, dst


def sgmm_edges(n, src, dst):
    """SGMM over the edge list (src[i], dst[i]) in list order.

    Returns (mate uint32[n], pairs uint32[k, 2]) with pairs in the order taken."""
    n, src, dst = _edges(n, src, dst)
    mate = np.empty(n, dtype=np.uint32)
    pairs = np.empty((max(n // 2, 1), 2), dtype=np.uint32)
    k = _load().oracle_sgmm_edges(n, src.size, _ptr(src), _ptr(dst), _ptr(mate), _ptr(pairs))
    if k < 0:
        raise ValueError("oracle_sgmm_edges failed (endpoint id out of range or no memory)")
    return mate, pairs[:k].copy()


def check_edges(n, src, dst, mate, pairs=None) -> Verdict:
    """Exact checker with the edge list as the edge set; first_uncovered is an
    index into the list."""
    n, src, dst = _edges(n, src, dst)
    mate = _u32(mate)
    if mate.size != n:
        raise ValueError("mate must have n entries")
    count = 0
    pp = None
    if pairs is not None:
        pairs = _u32(pairs).reshape(-1, 2)
        count = pairs.shape[0]
        if count == 0:
            pairs = np.zeros((1, 2), dtype=np.uint32)
        pp = _ptr(pairs)
    v = Verdict()
    rc = _load().oracle_check_edges(n, src.size, _ptr(src), _ptr(dst), _ptr(mate), pp, count,
                                    ctypes.byref(v))
    if rc != 0:
        raise MemoryError("oracle_check_edges: no memory")
    return v


def cpu_skipper(offsets, nbrs, threads: int, row_skip: bool = False, rows=None,
                block_edges: int = 1 << 16):
    """Algorithm 1 on `threads` host threads over rows [r0, r1) (default: all).

    Returns (mate uint32[n], seconds of the parallel pass, failed CAS count)."""
    offsets = np.ascontiguousarray(np.asarray(offsets), dtype=np.int64)
    nbrs = _u32(nbrs)
    n = offsets.size - 1
    r0, r1 = (0, n) if rows is None else (int(rows[0]), int(min(rows[1], n)))
    mate = np.empty(n, dtype=np.uint32)
    sec = ctypes.c_double(0.0)
    rc = _load().cpu_skipper(n, _ptr(offsets), _ptr(nbrs), r0, r1, int(threads), int(block_edges),
                             1 if row_skip else 0, _ptr(mate), ctypes.byref(sec))
    if rc == -2:
        raise RuntimeError("cpu_skipper: a wait ran past its bound")
    if rc < 0:
        raise RuntimeError("cpu_skipper: allocation or thread start failed")
    return mate, float(sec.value), int(rc)
