"""Skipper maximal matching on GB300 (sm_103a CUDA behind a C ABI).

Skipper (Koohi Esfahani, arXiv 2507.04420) resolves every edge of an
undirected graph once, with a just-in-time reservation on a per-vertex state
ACC -> RSVD -> MCHD (Section IV, Algorithm 1).  This package is a thin binding
over ``libskipper.so`` (``include/skipper.h``): it only marshals torch tensors
(device memory) and streams into the C calls.  Every step of the matching runs
in the library's kernels; if the library is missing, import fails.

Mate arrays are returned as ``torch.int32`` tensors that hold uint32 bits:
an unmatched vertex reads as -1 (0xFFFFFFFF).
"""
from __future__ import annotations

import collections
import contextlib
import ctypes
from typing import Optional

import torch

from . import _native
from ._native import GraphDesc, Options, Stats, Timing, Verdict

__all__ = ["EdgeList", "Graph", "device_address", "HostSession", "Multi", "SkipperError", "match", "validate", "Options", "Verdict", "Timing",
           "UNMATCHED", "lib", "options"]

UNMATCHED = 0xFFFFFFFF
V_RANGE, V_ASYM, V_NONEDGE, V_UNCOVERED, V_PAIRS = 1, 2, 4, 8, 16

lib = _native.load()


class SkipperError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib.mm_last_error().decode(errors="replace")
        super().__init__(f"{where}: {_native.STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = _native.STATUS.get(code, str(code))


def _check(code: int, where: str):
    if code != 0:
        raise SkipperError(code, where)


def options(**kw) -> Options:
    """mm_options with the library defaults, overridden by keyword fields."""
    o = Options()
    _check(lib.mm_default_options(ctypes.byref(o)), "mm_default_options")
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, int(v))
    return o


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _ptr(t: Optional[torch.Tensor]) -> Optional[ctypes.c_void_p]:
    return None if t is None else ctypes.c_void_p(int(t.data_ptr()))


def _need(t: torch.Tensor, name: str, dtypes):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be in CUDA device memory")
    if t.dtype not in dtypes:
        raise TypeError(f"{name} must have dtype in {dtypes}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


_U32 = tuple(d for d in (torch.int32, getattr(torch, "uint32", None)) if d is not None)

MM_CHECK_CSR, MM_HOST_MAPPED, MM_BATCH_LOCAL_IDS = 1, 2, 4


def _need_pinned(t: torch.Tensor, name: str, dtypes):
    """A host tensor in page-locked memory (read in place by the kernels)."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.is_cuda or not t.is_pinned():
        raise ValueError(f"{name} must be a page-locked (pinned) host tensor for host_mapped")
    if t.dtype not in dtypes:
        raise TypeError(f"{name} must have dtype in {dtypes}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Graph:
    """A CSR handle (mm_create_csr); borrows offsets/nbrs, which must outlive it.

    The CSR is in device memory, or with host_mapped=True in page-locked host
    memory that the kernels read in place (MM_HOST_MAPPED): a call then moves
    over the host link only the entries it reads."""

    def __init__(self, offsets: torch.Tensor, nbrs: torch.Tensor, check: bool = True, stream=None,
                 host_mapped: bool = False, local_ids: bool = False):
        if host_mapped:
            _need_pinned(offsets, "offsets", (torch.int64,))
            if nbrs.numel():   # an empty array is never read
                _need_pinned(nbrs, "nbrs", _U32)
            self.device = torch.device("cuda", torch.cuda.current_device())
        else:
            _need(offsets, "offsets", (torch.int64,))
            _need(nbrs, "nbrs", _U32)
            self.device = offsets.device
        self.offsets, self.nbrs = offsets, nbrs
        self.n = offsets.numel() - 1
        self.nnz = nbrs.numel()
        flags = ((MM_CHECK_CSR if check else 0) | (MM_HOST_MAPPED if host_mapped else 0) |
                 (MM_BATCH_LOCAL_IDS if local_ids else 0))
        h = ctypes.c_void_p()
        _check(lib.mm_create_csr(self.n, self.nnz, _ptr(offsets), _ptr(nbrs) if self.nnz else None,
                                 flags, _stream_ptr(stream), ctypes.byref(h)),
               "mm_create_csr")
        self._h = h

    # -- matching -------------------------------------------------------------
    def skipper(self, mate: Optional[torch.Tensor] = None, pairs: bool = False,
                cap: Optional[int] = None, stream=None, opts: Optional[Options] = None, **kw):
        """Run Skipper; returns mate (int32 view of uint32), plus (pairs, count) if asked."""
        o = opts if opts is not None else options(**kw)
        dev = self.device
        if mate is None:
            mate = torch.empty(self.n, dtype=torch.int32, device=dev)
        _need(mate, "mate", _U32)
        if mate.numel() != self.n:
            raise ValueError("mate must have n entries")
        d_pairs = d_count = None
        if pairs:
            cap = cap if cap is not None else max(self.n // 2, 1)
            d_pairs = torch.empty((cap, 2), dtype=torch.int32, device=dev)
            d_count = torch.zeros(1, dtype=torch.int64, device=dev)
        _check(lib.mm_skipper(self._h, ctypes.byref(o), _ptr(mate), _ptr(d_pairs),
                              cap if pairs else 0, _ptr(d_count), _stream_ptr(stream)),
               "mm_skipper")
        if pairs:
            return mate, d_pairs, d_count
        return mate

    def skipper_to_host(self, host_mate: torch.Tensor, mate: Optional[torch.Tensor] = None,
                        pieces: int = 8, stream=None, opts: Optional[Options] = None, **kw) -> torch.Tensor:
        """Run Skipper with the result copied into `host_mate` (page-locked,
        int32[n]) piece by piece while the pass runs (mm_skipper_to_host);
        `mate` is the device array it is computed in.  Returns host_mate."""
        o = opts if opts is not None else options(**kw)
        if mate is None:
            mate = torch.empty(self.n, dtype=torch.int32, device=self.device)
        _need(mate, "mate", _U32)
        if mate.numel() != self.n or host_mate.numel() != self.n:
            raise ValueError("mate and host_mate must have n entries")
        if host_mate.dtype not in _U32 or host_mate.is_cuda or not host_mate.is_contiguous():
            raise ValueError("host_mate must be a contiguous int32 host tensor")
        _check(lib.mm_skipper_to_host(self._h, ctypes.byref(o), _ptr(mate), ctypes.c_void_p(host_mate.data_ptr()),
                                      pieces, _stream_ptr(stream)),
               "mm_skipper_to_host")
        return host_mate

    def batched(self, vbase: torch.Tensor, ebase: torch.Tensor, mate: Optional[torch.Tensor] = None,
                graph_pairs: bool = False, stream=None, opts: Optional[Options] = None, **kw):
        """Batched Skipper over a block-diagonal packing (vbase/ebase int64[G+1] on device)."""
        _need(vbase, "vbase", (torch.int64,))
        _need(ebase, "ebase", (torch.int64,))
        o = opts if opts is not None else options(**kw)
        G = vbase.numel() - 1
        if mate is None:
            mate = torch.empty(self.n, dtype=torch.int32, device=self.device)
        _need(mate, "mate", _U32)
        gp = torch.empty(G, dtype=torch.int64, device=self.device) if graph_pairs else None
        _check(lib.mm_skipper_batched(self._h, G, _ptr(vbase), _ptr(ebase), ctypes.byref(o),
                                      _ptr(mate), _ptr(gp), _stream_ptr(stream)),
               "mm_skipper_batched")
        return (mate, gp) if graph_pairs else mate

    def validate_batched(self, vbase: torch.Tensor, ebase: torch.Tensor, mate: torch.Tensor,
                         stream=None) -> Verdict:
        """One verdict over every member graph of a packed batch (mm_validate_batched)."""
        _need(vbase, "vbase", (torch.int64,))
        _need(ebase, "ebase", (torch.int64,))
        _need(mate, "mate", _U32)
        v = Verdict()
        _check(lib.mm_validate_batched(self._h, vbase.numel() - 1, _ptr(vbase), _ptr(ebase), _ptr(mate),
                                       ctypes.byref(v), _stream_ptr(stream)), "mm_validate_batched")
        return v

    def autotune(self, stream=None, opts: Optional[Options] = None, **kw) -> Options:
        """Fastest checked settings for skipper() on this graph (mm_autotune)."""
        o = opts if opts is not None else options(**kw)
        scratch = torch.empty(max(self.n, 1), dtype=torch.int32, device=self.device)
        _check(lib.mm_autotune(self._h, _ptr(scratch), ctypes.byref(o), _stream_ptr(stream)), "mm_autotune")
        return o

    def autotune_batched(self, vbase: torch.Tensor, ebase: torch.Tensor, stream=None,
                         opts: Optional[Options] = None, **kw) -> Options:
        o = opts if opts is not None else options(**kw)
        scratch = torch.empty(self.n, dtype=torch.int32, device=self.device)
        _check(lib.mm_autotune_batched(self._h, vbase.numel() - 1, _ptr(vbase), _ptr(ebase),
                                       _ptr(scratch), ctypes.byref(o), _stream_ptr(stream)),
               "mm_autotune_batched")
        return o

    def sync(self, stream=None):
        _check(lib.mm_sync(self._h, _stream_ptr(stream)), "mm_sync")

    def validate(self, mate: torch.Tensor, pairs: Optional[torch.Tensor] = None,
                 count: Optional[int] = None, stream=None) -> Verdict:
        _need(mate, "mate", _U32)
        if pairs is not None:
            _need(pairs, "pairs", _U32)
            count = pairs.shape[0] if count is None else count
        v = Verdict()
        _check(lib.mm_validate(self._h, _ptr(mate), _ptr(pairs), count or 0, ctypes.byref(v),
                               _stream_ptr(stream)), "mm_validate")
        return v

    def stats(self, stream=None) -> dict:
        """Sweep statistics of the last skipper(stats=1) call (reads, JIT conflicts)."""
        st = Stats()
        _check(lib.mm_get_stats(self._h, ctypes.byref(st), _stream_ptr(stream)), "mm_get_stats")
        return st.as_dict()

    def state_census(self, stream=None) -> dict:
        """Counts of the states the last skipper() call left (mm_state_census):
        after a completed call no vertex is RSVD and MCHD is twice the pairs."""
        out = (ctypes.c_uint64 * 4)()
        _check(lib.mm_state_census(self._h, out, _stream_ptr(stream)), "mm_state_census")
        return {"acc": int(out[0]), "rsvd": int(out[1]), "mchd": int(out[2]), "other": int(out[3])}

    @staticmethod
    def _tdict(t) -> dict:
        return {"init_ms": t.init_ms, "sweep_ms": t.sweep_ms, "compact_ms": t.compact_ms,
                "total_ms": t.total_ms, "units": int(t.units)}

    def timing(self) -> dict:
        """Per-kernel times of the last call made with timing=1."""
        t = Timing()
        _check(lib.mm_get_timing(self._h, ctypes.byref(t)), "mm_get_timing")
        return self._tdict(t)

    def timing_history(self, max_calls: int = 256) -> list:
        """Per-kernel times of the latest timed calls (oldest first); clears them."""
        arr = (Timing * max_calls)()
        cnt = ctypes.c_uint32(0)
        _check(lib.mm_timing_history(self._h, arr, max_calls, ctypes.byref(cnt)),
               "mm_timing_history")
        return [self._tdict(arr[i]) for i in range(cnt.value)]

    def close(self):
        if getattr(self, "_h", None):
            lib.mm_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class EdgeList(Graph):
    """A device edge-list handle (mm_create_coo): edge i is {src[i], dst[i]},
    each edge listed once in either direction.  Borrows src/dst, which must
    outlive it.  skipper / validate / stats / timing work as on a CSR handle;
    the batched calls do not apply."""

    def __init__(self, n: int, src: torch.Tensor, dst: torch.Tensor, check: bool = True, stream=None,
                 host_mapped: bool = False):
        if host_mapped:
            _need_pinned(src, "src", _U32)
            _need_pinned(dst, "dst", _U32)
            self.device = torch.device("cuda", torch.cuda.current_device())
        else:
            _need(src, "src", _U32)
            _need(dst, "dst", _U32)
            self.device = src.device
        if src.dim() != 1 or src.shape != dst.shape:
            raise ValueError("src and dst must be 1-D tensors of the same length")
        self.src, self.dst = src, dst
        self.n = int(n)
        self.nnz = self.m = src.numel()
        flags = (MM_CHECK_CSR if check else 0) | (MM_HOST_MAPPED if host_mapped else 0)
        h = ctypes.c_void_p()
        _check(lib.mm_create_coo(self.n, self.m, _ptr(src) if self.m else None,
                                 _ptr(dst) if self.m else None, flags,
                                 _stream_ptr(stream), ctypes.byref(h)), "mm_create_coo")
        self._h = h


def match(offsets: torch.Tensor, nbrs: torch.Tensor, **kw) -> torch.Tensor:
    """One-shot Skipper on a device CSR; returns the mate array (int32 view of uint32)."""
    with Graph(offsets, nbrs) as g:
        return g.skipper(**kw)


def validate(offsets: torch.Tensor, nbrs: torch.Tensor, mate: torch.Tensor, pairs=None) -> Verdict:
    with Graph(offsets, nbrs, check=False) as g:
        return g.validate(mate, pairs)


def device_address(t: torch.Tensor) -> int:
    """Device address of a tensor's memory: its data pointer for a CUDA tensor,
    the in-place address (mm_host_device_address) for a host tensor."""
    if t.is_cuda:
        return t.data_ptr()
    out = ctypes.c_void_p()
    _check(lib.mm_host_device_address(ctypes.c_void_p(t.data_ptr()), ctypes.byref(out)),
           "mm_host_device_address")
    return int(out.value)


class Multi:
    """Many independent graphs, each in its own device tensors, matched in one
    launch (mm_skipper_multi) and checked in one launch (mm_validate_multi).

    A graph is a tuple (offsets int64[n+1], nbrs int32[nnz], mate int32[n]) of
    CUDA tensors; with allow_host=True offsets and nbrs may also be pinned
    host tensors, which the kernels read in place (the device addresses of
    page-locked memory are its host addresses under unified addressing).
    Calls on one Multi must be ordered (one stream)."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(lib.mm_multi_create(ctypes.byref(h)), "mm_multi_create")
        self._h = h

    @staticmethod
    def _descs(graphs, allow_host: bool = False):
        arr = (GraphDesc * max(1, len(graphs)))()
        for i, (off, nb, mate) in enumerate(graphs):
            if allow_host and not off.is_cuda:
                _need_pinned(off, "offsets", (torch.int64,))
                _need_pinned(nb, "nbrs", _U32)
            else:
                _need(off, "offsets", (torch.int64,))
                _need(nb, "nbrs", _U32)
            _need(mate, "mate", _U32)
            arr[i].n = off.numel() - 1
            arr[i].nnz = nb.numel()
            arr[i].offsets = device_address(off)
            arr[i].nbrs = device_address(nb) if nb.numel() else None
            arr[i].mate = mate.data_ptr() if mate.numel() else None
        return arr

    def run_descs(self, arr, count: int, stream=None, opts: Optional[Options] = None, **kw):
        """mm_skipper_multi over a GraphDesc array the caller filled (device addresses)."""
        o = opts if opts is not None else options(**kw)
        _check(lib.mm_skipper_multi(self._h, count, arr, ctypes.byref(o), _stream_ptr(stream)),
               "mm_skipper_multi")

    def validate_async_descs(self, arr, count: int, stream=None):
        _check(lib.mm_validate_multi_async(self._h, count, arr, _stream_ptr(stream)),
               "mm_validate_multi_async")

    def run(self, graphs, stream=None, opts: Optional[Options] = None, allow_host: bool = False, **kw):
        o = opts if opts is not None else options(**kw)
        arr = self._descs(graphs, allow_host)
        _check(lib.mm_skipper_multi(self._h, len(graphs), arr, ctypes.byref(o), _stream_ptr(stream)),
               "mm_skipper_multi")

    def sync(self, stream=None):
        _check(lib.mm_multi_sync(self._h, _stream_ptr(stream)), "mm_multi_sync")

    def validate(self, graphs, stream=None, allow_host: bool = False):
        arr = self._descs(graphs, allow_host)
        out = (Verdict * max(1, len(graphs)))()
        _check(lib.mm_validate_multi(self._h, len(graphs), arr, out, _stream_ptr(stream)),
               "mm_validate_multi")
        return [out[i] for i in range(len(graphs))]

    def validate_async(self, graphs, stream=None, allow_host: bool = False):
        """Enqueue the checker for these graphs on the stream (after a run on it)."""
        arr = self._descs(graphs, allow_host)
        _check(lib.mm_validate_multi_async(self._h, len(graphs), arr, _stream_ptr(stream)),
               "mm_validate_multi_async")

    def verdicts(self, count: int):
        """Verdicts of the last validate_async, once its stream has passed it."""
        out = (Verdict * max(1, count))()
        _check(lib.mm_multi_verdicts(self._h, count, out), "mm_multi_verdicts")
        return [out[i] for i in range(count)]

    def close(self):
        if getattr(self, "_h", None):
            lib.mm_multi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostSession:
    """Skipper on graphs that live in host memory.

    Two ways in.  zero_copy=True (the default) with page-locked (pinned) host
    tensors and no check: the kernels read the CSR in place through the host
    link (MM_HOST_MAPPED), so a run moves only the offsets and the neighbour
    ids the sweep reads -- on Grace-Blackwell over NVLink-C2C.  Otherwise
    (pageable tensors, zero_copy=False, or check=True, whose checker reads
    every entry and is better served by one bulk copy): the CSR is copied into
    device buffers kept for up to (n_max, nnz_max).  Either way the mate array
    is computed in device memory and copied back; read in place with
    pieces > 0, it comes back in that many parts while the pass runs
    (mm_skipper_to_host), unless the options ask for what that call does not
    run (dispersed units, serial mode, statistics, timing, a CUDA graph)."""

    HANDLES = 16   # handles kept per way in (least recently used first out)

    def __init__(self, n_max: int, nnz_max: int, device=None, zero_copy: bool = True, pieces: int = 0):
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.n_max, self.nnz_max = n_max, nnz_max
        self.zero_copy = zero_copy
        self.pieces = pieces
        self.dev = dev
        self.d_off = self.d_nb = None       # copy-path buffers, made on first use
        self.d_mate = torch.empty(max(n_max, 1), dtype=torch.int32, device=dev)
        self._graphs = collections.OrderedDict()   # copy-path handles, keyed by (n, nnz)
        self._mapped = collections.OrderedDict()   # host-mapped handles, keyed by the host arrays
        self.last_verdict = None
        self.last_mode = None
        self.last_pieces = 0   # > 0: the last run copied its result back in pieces

    def run(self, offsets: torch.Tensor, nbrs: torch.Tensor, mate_out: Optional[torch.Tensor] = None,
            stream=None, check: bool = False, **kw) -> torch.Tensor:
        n, nnz = offsets.numel() - 1, nbrs.numel()
        if n > self.n_max or nnz > self.nnz_max:
            raise ValueError("graph larger than the session's buffers")
        mate_d = self.d_mate[:n]
        # the copies are enqueued on the stream the calls run on
        with torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext():
            return self._run(offsets, nbrs, mate_out, stream, check, n, nnz, mate_d, **kw)

    def _run(self, offsets, nbrs, mate_out, stream, check, n, nnz, mate_d, **kw):
        self.last_pieces = 0
        if self.zero_copy and not check and offsets.is_pinned() and (nnz == 0 or nbrs.is_pinned()):
            self.last_mode = "host_mapped"
            key = (offsets.data_ptr(), nbrs.data_ptr(), n, nnz)
            g = self._mapped.get(key)
            if g is None:  # one handle per pair of host arrays (read in place)
                g = Graph(offsets, nbrs, check=False, stream=stream, host_mapped=True)
                self._mapped[key] = g
                while len(self._mapped) > self.HANDLES:
                    self._mapped.popitem(last=False)[1].close()
            self._mapped.move_to_end(key)
            o = kw.get("opts") or options(**{k: v for k, v in kw.items() if k != "opts"})
            if (self.pieces and o.unit_order != 2 and not o.serial and not o.stats and not o.timing
                    and not o.use_graph):
                if mate_out is None:
                    mate_out = torch.empty(n, dtype=torch.int32, pin_memory=True)
                if mate_out.is_pinned():
                    self.last_pieces = self.pieces
                    self.last_verdict = None
                    g.skipper_to_host(mate_out, mate=mate_d, pieces=self.pieces, stream=stream, opts=o)
                    (stream or torch.cuda.current_stream()).synchronize()
                    return mate_out
        else:
            self.last_mode = "copy"
            if self.d_off is None:
                self.d_off = torch.zeros(self.n_max + 1, dtype=torch.int64, device=self.dev)
                self.d_nb = torch.empty(max(self.nnz_max, 4), dtype=torch.int32, device=self.dev)
            off_d, nb_d = self.d_off[: n + 1], self.d_nb[:nnz]
            off_d.copy_(offsets, non_blocking=True)
            nb_d.copy_(nbrs, non_blocking=True)
            key = (n, nnz)
            g = self._graphs.get(key)
            if g is None:  # the handle only borrows the buffers; their contents change per run
                g = self._graphs[key] = Graph(off_d, nb_d, check=False, stream=stream)
                while len(self._graphs) > self.HANDLES:
                    self._graphs.popitem(last=False)[1].close()
            self._graphs.move_to_end(key)
        g.skipper(mate=mate_d, stream=stream, **kw)
        self.last_verdict = g.validate(mate_d, stream=stream) if check else None
        if mate_out is None:
            mate_out = torch.empty(n, dtype=torch.int32, pin_memory=True)
        mate_out.copy_(mate_d, non_blocking=True)
        (stream or torch.cuda.current_stream()).synchronize()
        return mate_out

    def close(self):
        for g in list(self._graphs.values()) + list(self._mapped.values()):
            g.close()
        self._graphs.clear()
        self._mapped.clear()
