"""Continuous-batching Skipper server on one GPU (binding of the native server).

The serving loop runs in the library (``mm_server_*`` in ``include/skipper.h``,
``csrc/server.cu``): one native worker thread admits requests in arrival
order while their device footprint fits the memory budget and, whenever a
compute slot is free, launches one multi-graph pass (mm_skipper_multi) over
every request admitted since the last launch, then the exact device checker
(mm_validate_multi) on the same stream.  Two compute slots alternate, so a new
batch is admitted and launched while the previous one is still on the GPU.

A request reaches the GPU one of two ways.  Small requests (up to
in_place_max_nnz entries) whose host arrays the device can address are read
in place through the host link, their mate arrays sharing one device arena per
launch; larger ones are copied to their own device buffers.  Each mate array
is copied back into the request's host buffer.

This module only marshals tensors: Server.submit hands the host arrays to the
native server and Request.wait collects the result (the wait runs in C, without
the interpreter lock).  Latency of a request = completion (mate in host
memory, verdict known) minus submission, both on the monotonic clock that
time.perf_counter() reads.
"""
from __future__ import annotations

import ctypes
import threading
import time
from typing import Dict, List, Optional, Sequence, Tuple

import torch

from . import SkipperError, lib, options
from ._native import ServerConfig, ServerResult, Verdict

__all__ = ["Request", "Server", "device_bytes", "plan_admission"]

MM_OK, MM_ERR_OOM, MM_PENDING = 0, 2, 7


def _ok(code: int, where: str):
    if code != MM_OK:
        raise SkipperError(code, where)


def device_bytes(n: int, nnz: int, in_place: bool = False) -> int:
    """Device memory a request holds while resident (mm_server_device_bytes):
    its CSR unless read in place, its mate, and its share of the launch scratch
    (packed states, partition and unit tables, the checker's marks)."""
    out = ctypes.c_uint64()
    _ok(lib.mm_server_device_bytes(n, nnz, 1 if in_place else 0, ctypes.byref(out)), "mm_server_device_bytes")
    return int(out.value)


def plan_admission(sizes: Sequence[int], used: int, budget: int, max_graphs: int) -> Tuple[int, int]:
    """How many of the pending requests (sizes in bytes, arrival order) to admit
    (mm_server_plan_admission): in arrival order, stopping at the first that
    does not fit (no overtaking, so no request starves).  Returns (count, bytes)."""
    arr = (ctypes.c_uint64 * max(1, len(sizes)))(*sizes)
    k, add = ctypes.c_uint64(), ctypes.c_uint64()
    _ok(lib.mm_server_plan_admission(arr, len(sizes), used, budget, max_graphs, ctypes.byref(k),
                                     ctypes.byref(add)), "mm_server_plan_admission")
    return int(k.value), int(add.value)


class Request:
    __slots__ = ("rid", "offsets", "nbrs", "n", "nnz", "arrival", "done_t", "mate", "verdict",
                 "error", "in_place", "_server", "_lock")

    def __init__(self, server: "Server", offsets: torch.Tensor, nbrs: torch.Tensor, mate: torch.Tensor):
        self.rid = 0
        self.offsets, self.nbrs, self.mate = offsets, nbrs, mate   # kept alive until collected
        self.n, self.nnz = offsets.numel() - 1, nbrs.numel()
        self.arrival = time.perf_counter()
        self.done_t = None
        self.verdict = None
        self.error = None
        self.in_place = None
        self._server = server
        self._lock = threading.Lock()

    def wait(self, timeout: Optional[float] = None) -> bool:
        """Wait for the result (True once it is in: mate, verdict, error set)."""
        if self.done_t is not None:
            return True
        return self._server._collect(self, 1e9 if timeout is None else timeout)

    @property
    def latency(self) -> Optional[float]:
        return None if self.done_t is None else self.done_t - self.arrival


class Server:
    def __init__(self, device=None, memory_bytes: Optional[int] = None, reserve_bytes: int = 8 << 30,
                 max_graphs_per_tick: int = 4096, max_bytes_per_tick: int = 32 << 30,
                 status_bits: int = 32, grain: int = 2048, serial: bool = False,
                 validate: bool = True, slots: int = 2, in_place_max_nnz: int = 1 << 20):
        self.dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        cfg = ServerConfig()
        _ok(lib.mm_server_default_config(ctypes.byref(cfg)), "mm_server_default_config")
        cfg.memory_bytes = 0 if memory_bytes is None else int(memory_bytes)
        cfg.reserve_bytes = reserve_bytes
        cfg.max_graphs_per_tick = max_graphs_per_tick
        cfg.max_bytes_per_tick = max_bytes_per_tick
        cfg.in_place_max_nnz = in_place_max_nnz
        cfg.validate = 1 if validate else 0
        cfg.slots = slots
        cfg.opts = options(status_bits=status_bits, grain=grain, serial=int(serial), nosync=1)
        self.validate = validate
        h = ctypes.c_void_p()
        with torch.cuda.device(self.dev):
            _ok(lib.mm_server_create(ctypes.byref(cfg), ctypes.byref(h)), "mm_server_create")
        self._h = h
        if memory_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.dev)
            self.budget = max(0, free - reserve_bytes)
        else:
            self.budget = int(memory_bytes)
        self._live: Dict[int, Request] = {}
        self._lock = threading.Lock()
        self.ticks = 0
        self.graphs_launched = 0
        self.error: Optional[BaseException] = None

    # -- client side ------------------------------------------------------------
    def submit(self, offsets: torch.Tensor, nbrs: torch.Tensor,
               mate_out: Optional[torch.Tensor] = None) -> Request:
        """Queue one graph (host CSR; page-locked memory makes the copies
        asynchronous and small requests eligible for reading in place).

        mate_out: optional host int32 tensor of n entries (page-locked for an
        asynchronous copy) that receives the result; a client that recycles
        its result buffers keeps pinned allocations out of the serving loop.
        Without it the server allocates one."""
        if offsets.is_cuda or nbrs.is_cuda:
            raise ValueError("submit host tensors")
        if offsets.dtype != torch.int64 or nbrs.dtype != torch.int32:
            raise TypeError("offsets must be int64 and nbrs int32 (uint32 bits)")
        if not (offsets.is_contiguous() and nbrs.is_contiguous()):
            raise ValueError("offsets and nbrs must be contiguous")
        n = offsets.numel() - 1
        if mate_out is None:
            mate_out = torch.empty(n, dtype=torch.int32, pin_memory=True)
        elif (mate_out.is_cuda or mate_out.numel() != n or mate_out.dtype != torch.int32
              or not mate_out.is_contiguous()):
            raise ValueError("mate_out must be a contiguous host int32 tensor of n entries")
        req = Request(self, offsets, nbrs, mate_out)
        ticket = ctypes.c_uint64()
        rc = lib.mm_server_submit(self._h, n, nbrs.numel(), ctypes.c_void_p(offsets.data_ptr()),
                                  ctypes.c_void_p(nbrs.data_ptr()) if nbrs.numel() else None,
                                  ctypes.c_void_p(mate_out.data_ptr()) if n else None, ctypes.byref(ticket))
        if rc != MM_OK:
            req.error = SkipperError(rc, "mm_server_submit")
            req.done_t = time.perf_counter()
            return req
        req.rid = int(ticket.value)
        with self._lock:
            self._live[req.rid] = req
        return req

    def _collect(self, req: Request, timeout: float) -> bool:
        with req._lock:
            if req.done_t is not None:
                return True
            res = ServerResult()
            rc = lib.mm_server_wait(self._h, req.rid, float(timeout), ctypes.byref(res))
            if rc == MM_PENDING:
                return False
            _ok(rc, "mm_server_wait")
            req.in_place = bool(res.in_place)
            req.arrival = res.submit_ns * 1e-9
            if res.status == MM_OK:
                if self.validate:
                    v = Verdict()
                    ctypes.memmove(ctypes.byref(v), ctypes.byref(res.verdict), ctypes.sizeof(Verdict))
                    req.verdict = v
            elif res.status == MM_ERR_OOM:
                req.error = MemoryError(f"request needs {device_bytes(req.n, req.nnz, req.in_place)} "
                                        f"device bytes, budget {self.budget}")
            else:
                req.error = SkipperError(res.status, "server request")
            req.done_t = res.done_ns * 1e-9
        with self._lock:
            self._live.pop(req.rid, None)
        return True

    def stats(self) -> Tuple[int, int, int]:
        """(launches, graphs launched, device bytes held by admitted requests)."""
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _ok(lib.mm_server_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "mm_server_stats")
        return int(a.value), int(b.value), int(c.value)

    @property
    def tick_sizes(self) -> List[float]:
        """Mean graphs per launch, as a one-element list (the native server keeps totals)."""
        return [self.graphs_launched / self.ticks] if self.ticks else [0.0]

    def close(self, timeout: float = 600.0):
        """Collect every outstanding result, then stop the native server."""
        if not getattr(self, "_h", None):
            return
        with self._lock:
            live = list(self._live.values())
        for r in live:
            r.wait(timeout)
        self.ticks, self.graphs_launched, _ = self.stats()
        rc = lib.mm_server_destroy(self._h)
        self._h = None
        if rc != MM_OK:
            self.error = SkipperError(rc, "mm_server_destroy")
            raise self.error

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
