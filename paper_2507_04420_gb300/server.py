"""Continuous-batching Skipper server on one GPU.

Requests (graphs in host memory) arrive at any time.  A worker thread admits
them in arrival order while their device footprint fits the memory budget and
whenever a compute slot is free launches one multi-graph pass
(mm_skipper_multi) over every request admitted since the last launch.  Two
compute slots alternate, so a new batch is admitted and launched while the
previous one is still on the GPU.  Each result is checked by the exact device
checker (mm_validate_multi) before its request completes; its mate array is
copied back on a second copy stream.

A request reaches the GPU one of two ways.  Small requests in page-locked
memory (up to in_place_max_nnz entries) are read in place: the kernels read
their CSR through the host link (their device addresses come from
mm_host_device_address on the client thread), and their mate arrays share one
device arena per launch -- no device allocation and no host->device copy per
request.  Larger ones are copied to their own device buffers on a copy stream
(their checker reads every entry, which one bulk copy serves best); the CSR and
the state stay resident until the request completes.

Latency of a request = completion (mate in host memory, verdict known) minus
submission.
"""
from __future__ import annotations

import collections
import queue
import threading
import time
from typing import List, Optional, Sequence, Tuple

import torch

from . import GraphDesc, Multi, SkipperError, device_address, options

__all__ = ["Request", "Server", "device_bytes", "plan_admission"]


def device_bytes(n: int, nnz: int, in_place: bool = False) -> int:
    """Device memory a request holds while resident: offsets and neighbour ids
    (not when read in place), mate, plus its share of the launch scratch
    (packed states, partition and unit tables, the checker's marks), rounded
    up to 512-byte granules."""
    r = lambda b: (b + 511) // 512 * 512
    scratch = (n // 4 + 8) + n + 24 * ((n + nnz) // 1024 + 2)
    csr = 0 if in_place else r(8 * (n + 1)) + r(4 * max(nnz, 1))
    return csr + r(4 * max(n, 1)) + r(scratch)


def plan_admission(sizes: Sequence[int], used: int, budget: int, max_graphs: int) -> Tuple[int, int]:
    """How many of the pending requests (sizes in bytes, arrival order) to admit.

    Admission is in arrival order and stops at the first request that does not
    fit (no overtaking, so no request starves).  Returns (count, bytes)."""
    k = 0
    add = 0
    for s in sizes:
        if k >= max_graphs or used + add + s > budget:
            break
        add += s
        k += 1
    return k, add


class Request:
    __slots__ = ("rid", "offsets", "nbrs", "n", "nnz", "arrival", "done_t", "mate", "verdict",
                 "error", "in_place", "_event", "_dev", "_addr", "_mate_d", "_bytes", "tick")

    def __init__(self, rid: int, offsets: torch.Tensor, nbrs: torch.Tensor, in_place: bool = False):
        self.rid = rid
        self.offsets, self.nbrs = offsets, nbrs
        self.n, self.nnz = offsets.numel() - 1, nbrs.numel()
        self.arrival = time.perf_counter()
        self.done_t = None
        self.mate = None
        self.verdict = None
        self.error = None
        self.in_place = in_place
        self._event = threading.Event()
        self._dev = None
        self._addr = None      # (offsets, nbrs) device addresses when read in place
        self._mate_d = None    # device mate (a slice of the launch's arena when read in place)
        self._bytes = device_bytes(self.n, self.nnz, in_place)
        self.tick = None

    def wait(self, timeout: Optional[float] = None) -> bool:
        return self._event.wait(timeout)

    @property
    def latency(self) -> Optional[float]:
        return None if self.done_t is None else self.done_t - self.arrival


class Server:
    def __init__(self, device=None, memory_bytes: Optional[int] = None, reserve_bytes: int = 8 << 30,
                 max_graphs_per_tick: int = 4096, max_bytes_per_tick: int = 32 << 30,
                 status_bits: int = 32, grain: int = 2048, serial: bool = False,
                 validate: bool = True, slots: int = 2, in_place_max_nnz: int = 1 << 20):
        self.dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        free, _ = torch.cuda.mem_get_info(self.dev)
        self.budget = memory_bytes if memory_bytes is not None else max(0, free - reserve_bytes)
        self.max_graphs = max_graphs_per_tick
        self.max_tick_bytes = max_bytes_per_tick
        self.validate = validate
        self.in_place_max_nnz = in_place_max_nnz
        self.opts = options(status_bits=status_bits, grain=grain, serial=int(serial), nosync=1)
        self.h2d = torch.cuda.Stream(self.dev)
        self.d2h = torch.cuda.Stream(self.dev)
        self.slots = [(torch.cuda.Stream(self.dev), Multi()) for _ in range(slots)]
        self._next_slot = 0
        self._inbox: "queue.Queue[Request]" = queue.Queue()
        self._rid = 0
        self._lock = threading.Lock()
        self._closing = False
        self.used = 0
        self.ticks = 0
        self.tick_sizes: List[int] = []
        self.error: Optional[BaseException] = None
        self._thread = threading.Thread(target=self._run, name="skipper-server", daemon=True)
        self._thread.start()

    # -- client side ------------------------------------------------------------
    def submit(self, offsets: torch.Tensor, nbrs: torch.Tensor,
               mate_out: Optional[torch.Tensor] = None) -> Request:
        """Queue one graph (host CSR; pinned memory makes the copy asynchronous).

        mate_out: optional host int32 tensor of n entries (pinned for an
        asynchronous copy) that receives the result; a client that recycles
        its result buffers keeps pinned allocations out of the serving loop.
        Without it the server allocates one."""
        if offsets.is_cuda or nbrs.is_cuda:
            raise ValueError("submit host tensors")
        if mate_out is not None and (mate_out.is_cuda or mate_out.numel() != offsets.numel() - 1
                                     or mate_out.dtype != torch.int32):
            raise ValueError("mate_out must be a host int32 tensor of n entries")
        with self._lock:
            rid = self._rid
            self._rid += 1
        nnz = nbrs.numel()
        in_place = (nnz <= self.in_place_max_nnz and offsets.is_pinned() and (nnz == 0 or nbrs.is_pinned())
                    and offsets.dtype == torch.int64 and nbrs.dtype in (torch.int32,)
                    and offsets.is_contiguous() and nbrs.is_contiguous())
        req = Request(rid, offsets, nbrs, in_place)
        if in_place:   # resolved here, on the client thread
            req._addr = (device_address(offsets), device_address(nbrs) if nnz else 0)
        req.mate = mate_out
        if self.error is not None:
            req.error = self.error
            req.done_t = time.perf_counter()
            req._event.set()
            return req
        if req._bytes > self.budget:
            req.error = MemoryError(f"request needs {req._bytes} device bytes, budget {self.budget}")
            req.done_t = time.perf_counter()
            req._event.set()
            return req
        self._inbox.put(req)
        return req

    def close(self, timeout: float = 600.0):
        self._closing = True
        self._thread.join(timeout)
        for _, m in self.slots:
            m.close()
        if self.error is not None:
            raise self.error

    # -- worker -------------------------------------------------------------------
    def _admit(self, req: Request):
        if req.in_place:       # its mate is carved from the launch's arena
            return
        with torch.cuda.stream(self.h2d):
            off = torch.empty(req.n + 1, dtype=torch.int64, device=self.dev)
            nb = torch.empty(max(req.nnz, 1), dtype=torch.int32, device=self.dev)[: req.nnz]
            mate = torch.empty(req.n, dtype=torch.int32, device=self.dev)
            off.copy_(req.offsets, non_blocking=True)
            if req.nnz:
                nb.copy_(req.nbrs, non_blocking=True)
        req._dev = (off, nb, mate)
        req._mate_d = mate

    def _launch(self, batch: List[Request]):
        stream, multi = self.slots[self._next_slot]
        slot = self._next_slot
        self._next_slot = (self._next_slot + 1) % len(self.slots)
        copied = torch.cuda.Event()
        copied.record(self.h2d)
        stream.wait_event(copied)
        arena = None
        total = sum(r.n for r in batch if r.in_place)
        if total:  # one device allocation for the mates of all in-place requests
            with torch.cuda.stream(stream):
                arena = torch.empty(total, dtype=torch.int32, device=self.dev)
            at = 0
            for r in batch:
                if r.in_place:
                    r._mate_d = arena[at:at + r.n]
                    at += r.n
        arr = (GraphDesc * max(1, len(batch)))()
        for i, r in enumerate(batch):
            d = arr[i]
            d.n, d.nnz = r.n, r.nnz
            if r.in_place:
                d.offsets, d.nbrs = r._addr[0], (r._addr[1] or None)
            else:
                d.offsets, d.nbrs = r._dev[0].data_ptr(), (r._dev[1].data_ptr() if r.nnz else None)
            d.mate = r._mate_d.data_ptr() if r.n else None
        multi.run_descs(arr, len(batch), stream=stream, opts=self.opts)
        swept = torch.cuda.Event()
        swept.record(stream)
        if self.validate:  # the checker runs behind the pass, on the same stream
            multi.validate_async_descs(arr, len(batch), stream=stream)
        checked = torch.cuda.Event()
        checked.record(stream)
        for r in batch:  # the device tensors were made on the copy stream; they are used here too
            if r._dev is not None:
                for t in r._dev:
                    t.record_stream(stream)
        self.d2h.wait_event(swept)
        with torch.cuda.stream(self.d2h):
            for r in batch:
                if r.mate is None:
                    r.mate = torch.empty(r.n, dtype=torch.int32, pin_memory=True)
                r.mate.copy_(r._mate_d, non_blocking=True)
            if arena is not None:
                arena.record_stream(self.d2h)
            for r in batch:
                if r._dev is not None:
                    r._dev[2].record_stream(self.d2h)
        back = torch.cuda.Event()
        back.record(self.d2h)
        self.ticks += 1
        self.tick_sizes.append(len(batch))
        return (slot, batch, back, checked)

    def _complete(self, tick) -> bool:
        slot, batch, back, checked = tick
        if not (back.query() and checked.query()):
            return False
        stream, multi = self.slots[slot]
        err = None
        try:
            multi.sync(stream)  # the pass's own status (timeouts, bad ids)
        except SkipperError as e:
            err = e
        verdicts = multi.verdicts(len(batch)) if (self.validate and err is None) else None
        now = time.perf_counter()
        for i, r in enumerate(batch):
            r.verdict = None if verdicts is None else verdicts[i]
            r.error = err
            r.done_t = now
            r._dev = None
            r._mate_d = None
            self.used -= r._bytes
            r._event.set()
        return True

    def _run(self):
        pending: "collections.deque[Request]" = collections.deque()
        staged: List[Request] = []
        inflight: "collections.deque" = collections.deque()
        torch.cuda.set_device(self.dev)
        try:
            while True:
                busy = False
                while True:
                    try:
                        pending.append(self._inbox.get_nowait())
                    except queue.Empty:
                        break
                while inflight and self._complete(inflight[0]):
                    inflight.popleft()
                    busy = True
                staged_bytes = sum(r._bytes for r in staged)
                room = min(self.budget, self.used + self.max_tick_bytes - staged_bytes)
                k, add = plan_admission([r._bytes for r in pending], self.used, room,
                                        self.max_graphs - len(staged))
                if k == 0 and not staged and not inflight and pending and pending[0]._bytes > self.max_tick_bytes:
                    k, add = 1, pending[0]._bytes  # one request larger than a tick runs alone
                for _ in range(k):
                    r = pending.popleft()
                    self._admit(r)
                    staged.append(r)
                    busy = True
                self.used += add
                if staged and len(inflight) < len(self.slots):
                    inflight.append(self._launch(staged))
                    staged = []
                    busy = True
                if self._closing and not pending and not staged and not inflight and self._inbox.empty():
                    return
                if not busy:
                    time.sleep(50e-6)
        except BaseException as e:  # surface worker failures to close() and to every waiter
            self.error = e
            self._closing = True
            left = list(pending) + staged + [r for t in inflight for r in t[1]]
            while True:
                try:
                    left.append(self._inbox.get_nowait())
                except queue.Empty:
                    break
            for r in left:
                r.error = e
                r.done_t = time.perf_counter()
                r._event.set()
