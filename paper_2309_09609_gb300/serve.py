"""Serving loop: a resident database, memory-bounded admission and continuous
batching over a pool of CUDA-stream slots.

The search itself is the library's (``sw_plan_search_async``); this module
only schedules it.  A request is one query; its result is the exact score
row against every subject.

* The database stays resident on the device for the life of the server.
* Admission: a request holds device memory while its batch runs: its scores
  row (4 bytes x subjects), allocated when the batch is launched and freed
  once the row is on the host, and its residues in the plan's query buffer.
  A request is admitted while the bytes of all admitted, unfinished requests
  stay within ``memory_budget``.  By default that is the smaller of what the
  slots can hold with every batch full and 90% of the device memory free
  when the server starts, so on a device that other work fills up, fewer
  requests run at once.  A request that could never fit is refused at once
  (``AdmissionError``), never queued forever.
* Continuous batching: a scheduler thread takes the admitted requests that
  have arrived, up to ``max_batch`` queries and ``max_batch_residues``
  residues, and launches them as one batch on a free slot (its own plan and
  CUDA stream).  Requests arriving while earlier batches run go to the next
  free slot, so batches of different lengths overlap on the GPU.  Two
  slots is the default: one batch's kernels run while the next batch is
  formed, staged and launched behind it.  More slots only queue on the GPU,
  because each search's persistent kernels occupy every SM.  On the
  570,000-subject database at 50 queries/s, 2 slots measured p50 77 ms and
  p99 185 ms, against 101 ms and 274 ms with 4 slots.
* Completion is observed per slot; each request gets its scores, its
  latency (arrival to completion on the host) and the batch it rode in.
* Cancellation: ``submit`` returns a ``concurrent.futures.Future``.
  Cancelling it before its batch is launched drops the request, which is then
  never admitted or searched.  Once launched it is running and can no longer
  be cancelled, as for any Future.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

from . import swgb


class AdmissionError(RuntimeError):
    """The request needs more memory than the server's whole budget."""


@dataclass
class Request:
    rid: int
    query: np.ndarray
    arrival: float
    future: Future = field(default_factory=Future)
    admitted: float = 0.0
    started: float = 0.0
    finished: float = 0.0
    batch: int = -1

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class _Slot:
    """One batch in flight: a plan, a CUDA stream and the batch's scores.

    The scheduler talks to a slot only through ``launch``, ``poll``,
    ``rows`` and ``close`` (and ``bind_thread`` once, on its own thread).
    The scores buffer is allocated per batch, at its size, and released by
    ``rows``, so the device memory a slot holds follows the admitted load."""

    def __init__(self, db, max_batch, max_residues, opts):
        import torch
        self.device = db.device
        self.n = db.n
        self.plan = db.plan(max_batch, max_residues, **opts)
        self.stream = torch.cuda.Stream(device=db.device)
        self.scores = None
        self.requests: list[Request] = []
        self.batch_id = -1

    @staticmethod
    def free_device_bytes(device) -> int:
        import torch
        return int(torch.cuda.mem_get_info(device)[0])

    @property
    def busy(self) -> bool:
        return bool(self.requests)

    def bind_thread(self):
        import torch
        torch.cuda.set_device(self.device)

    def launch(self, queries, lengths, gap_open, gap_extend, matrix):
        """Queues the batch's search on the slot's stream."""
        import torch
        with torch.cuda.stream(self.stream):   # allocated for use on this stream
            self.scores = torch.empty((lengths.size, self.n), dtype=torch.int32,
                                      device=f"cuda:{self.device}")
        try:
            self.plan.search_async(queries, lengths, self.scores, gap_open, gap_extend, matrix,
                                   stream=self.stream)
        except Exception:
            self.scores = None                   # nothing was queued: release the rows
            raise

    def poll(self) -> bool:
        """True once the batch's scores are complete (raises if it failed)."""
        return self.plan.wait(0)

    def rows(self, n) -> np.ndarray:
        """The finished batch's first n score rows, on the host; the device
        buffer is released."""
        try:
            return self.scores[:n].cpu().numpy()
        finally:
            self.scores = None

    def close(self):
        self.plan.close()


class Server:
    """Continuous-batching search server over one resident Database."""

    def __init__(self, db: swgb.Database, slots: int = 2, max_batch: int = 16,
                 max_batch_residues: int = 65536, memory_budget: int | None = None,
                 gap_open: int = 10, gap_extend: int = 2, matrix=None, slot_factory=None,
                 free_bytes=None, **plan_opts):
        """``slot_factory(db, max_batch, max_batch_residues, plan_opts)`` makes
        one slot (default: a plan and a stream on the GPU).  ``free_bytes()``
        gives the device memory free at start (default: the CUDA driver's
        figure with the default slots, no limit with a slot factory)."""
        self.db = db
        self.max_batch = int(max_batch)
        self.max_batch_residues = int(max_batch_residues)
        self.gap_open, self.gap_extend, self.matrix = gap_open, gap_extend, matrix
        make = slot_factory or _Slot
        self.slots = [make(db, self.max_batch, self.max_batch_residues, plan_opts)
                      for _ in range(int(slots))]
        if free_bytes is None and slot_factory is None:
            free_bytes = lambda: _Slot.free_device_bytes(db.device)  # noqa: E731
        # default: what the slots hold with every batch full (max_batch score
        # rows and max_batch_residues residues each), within 90% of the
        # device memory free now that the slots' plans exist
        full = len(self.slots) * (self.max_batch * self.request_bytes(0) + self.max_batch_residues)
        self.free_at_start = int(free_bytes()) if free_bytes else None
        if memory_budget:
            self.memory_budget = int(memory_budget)
        elif self.free_at_start is not None:
            self.memory_budget = min(full, int(0.9 * self.free_at_start))
        else:
            self.memory_budget = full
        self._lock = threading.Condition()
        self._pending: collections.deque[Request] = collections.deque()
        self._in_use = 0
        self.max_in_use = 0           # most bytes admitted at once
        self._next_id = 0
        self._batches = 0
        self.max_concurrent = 0       # most batches in flight at once
        self.cancelled = 0            # requests cancelled before they were launched
        self._stop = False
        self.completed: list[Request] = []
        self._thread = threading.Thread(target=self._loop, daemon=True)
        self._thread.start()

    # ---- admission ------------------------------------------------------------
    def request_bytes(self, query_len: int) -> int:
        """Device bytes a request holds while admitted: its scores row and its
        residues in the query buffer.  (The plan's border scratch and its
        bounded saturation list are allocated once per slot, whatever the
        load.)"""
        return 4 * self.db.n + int(query_len)

    def submit(self, query, arrival: float | None = None) -> Future:
        q = np.ascontiguousarray(query, dtype=np.uint8)
        if q.size and int(q.max()) >= 24:
            raise ValueError("residue codes must be 0..23")
        need = self.request_bytes(q.size)
        if need > self.memory_budget or q.size > self.max_batch_residues:
            raise AdmissionError(f"request needs {need} bytes / {q.size} residues; budget "
                                 f"{self.memory_budget} bytes / {self.max_batch_residues} residues")
        with self._lock:
            if self._stop:
                raise RuntimeError("server is closed")
            r = Request(self._next_id, q, time.perf_counter() if arrival is None else arrival)
            self._next_id += 1
            self._pending.append(r)
            self._lock.notify_all()
        return r.future

    # ---- scheduler ---------------------------------------------------------------
    def _take_batch(self):
        """Admitted requests for one batch (called with the lock held).  A
        request cancelled while it waited is dropped here; the ones taken are
        marked running, so from then on they can no longer be cancelled."""
        batch, residues = [], 0
        while self._pending and len(batch) < self.max_batch:
            r = self._pending[0]
            if r.future.cancelled():
                self._pending.popleft()
                self.cancelled += 1
                continue
            need = self.request_bytes(r.query.size)
            if residues + r.query.size > self.max_batch_residues:
                break
            if self._in_use + need > self.memory_budget:
                break
            self._pending.popleft()
            if not r.future.set_running_or_notify_cancel():   # cancelled just now
                self.cancelled += 1
                continue
            self._in_use += need
            self.max_in_use = max(self.max_in_use, self._in_use)
            r.admitted = time.perf_counter()
            batch.append(r)
            residues += r.query.size
        return batch

    def _launch(self, slot: _Slot, batch: list[Request]):
        q = np.concatenate([r.query for r in batch]) if batch else np.zeros(0, np.uint8)
        lens = np.array([r.query.size for r in batch], dtype=np.int32)
        now = time.perf_counter()
        for r in batch:
            r.started = now
            r.batch = self._batches
        slot.batch_id = self._batches
        self._batches += 1
        slot.requests = batch
        slot.launch(q, lens, self.gap_open, self.gap_extend, self.matrix)
        self.max_concurrent = max(self.max_concurrent, sum(s.busy for s in self.slots))

    def _fail(self, slot, batch, e):
        """A batch that failed fails its own requests only; its memory is released."""
        with self._lock:
            for r in batch:
                self._in_use -= self.request_bytes(r.query.size)
            slot.requests = []
            self._lock.notify_all()
        for r in batch:
            r.future.set_exception(e)

    def _complete(self, slot: _Slot):
        batch = slot.requests
        try:
            rows = slot.rows(len(batch))  # the slot's stream has finished
        except Exception as e:  # the copy to the host failed: like a failed search
            self._fail(slot, batch, e)
            return
        now = time.perf_counter()
        with self._lock:
            for i, r in enumerate(batch):
                r.finished = now
                self._in_use -= self.request_bytes(r.query.size)
                self.completed.append(r)
            slot.requests = []
            self._lock.notify_all()
        for i, r in enumerate(batch):
            r.future.set_result(rows[i].copy())

    def _loop(self):
        if self.slots:
            self.slots[0].bind_thread()
        while True:
            progressed = False
            for s in self.slots:
                if s.busy:
                    try:
                        done = s.poll()
                    except Exception as e:  # a failed batch fails its requests only
                        self._fail(s, s.requests, e)
                        progressed = True
                        continue
                    if done:
                        self._complete(s)
                        progressed = True
            with self._lock:
                if self._stop and not self._pending and not any(s.busy for s in self.slots):
                    return
                free = [s for s in self.slots if not s.busy]
                batch = self._take_batch() if free and self._pending else []
            if batch:
                try:
                    self._launch(free[0], batch)
                except Exception as e:
                    self._fail(free[0], batch, e)
                progressed = True
            if not progressed:
                with self._lock:
                    self._lock.wait(0.0002)

    def close(self, timeout: float = 600.0):
        with self._lock:
            self._stop = True
            self._lock.notify_all()
        self._thread.join(timeout)
        for s in self.slots:
            s.close()

    # ---- reporting --------------------------------------------------------------
    def report(self, wall_s: float | None = None) -> dict:
        lat = np.array([r.latency for r in self.completed]) * 1e3
        cells = sum(r.query.size for r in self.completed) * self.db.residues
        if wall_s is None and self.completed:
            wall_s = max(r.finished for r in self.completed) - min(r.arrival for r in self.completed)
        return {"requests": len(self.completed), "batches": self._batches,
                "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
                "mean_batch": len(self.completed) / max(self._batches, 1),
                "max_concurrent_batches": self.max_concurrent, "cancelled": self.cancelled,
                "memory_budget": self.memory_budget, "max_admitted_bytes": self.max_in_use,
                "gcups": cells / wall_s / 1e9 if wall_s else None, "wall_s": wall_s}


def replay(server: Server, arrivals, speed: float = 1.0, timeout: float = 600.0):
    """Submits a trace (synth.Arrivals) at its arrival times; returns futures."""
    t0 = time.perf_counter()
    futs = []
    for i in range(len(arrivals.queries)):
        target = t0 + arrivals.times[i] / speed
        delay = target - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        futs.append(server.submit(arrivals.queries.seq(i), arrival=max(target, t0)))
    for f in futs:
        f.result(timeout)
    return futs
