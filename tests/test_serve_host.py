"""The serving loop's scheduler on the CPU, with fake slots in place of GPU
plans: continuous batching within the batch limits and in arrival order,
memory-bounded admission, failures that stay with their own batch, and a
close that drains every admitted request."""
import threading
import time
import types

import numpy as np
import pytest

from paper_2309_09609_gb300 import serve

N_SUBJECTS = 7


def row_of(query):
    """The fake search's result for one query: identifies the query."""
    return np.arange(N_SUBJECTS, dtype=np.int32) + 1000 * int(query.size) + int(query.sum())


class Gate:
    """Holds every fake batch until the test opens it."""

    def __init__(self, open_=False):
        self.event = threading.Event()
        if open_:
            self.event.set()


class FakeSlot:
    log = None          # the query lengths of every launched batch, in launch order

    def __init__(self, gate, fail_launch=None, fail_poll=None, fail_rows=None):
        self.gate, self.fail_launch, self.fail_poll = gate, fail_launch, fail_poll
        self.fail_rows = fail_rows
        self.requests = []
        self.batch_id = -1
        self.rows_ = None
        self.lens = None

    @property
    def busy(self):
        return bool(self.requests)

    def bind_thread(self):
        pass

    def launch(self, queries, lengths, gap_open, gap_extend, matrix):
        assert lengths.dtype == np.int32 and int(lengths.sum()) == queries.size
        if self.fail_launch is not None and self.fail_launch in lengths.tolist():
            raise RuntimeError("launch failed")
        offs = np.concatenate([[0], np.cumsum(lengths)])
        self.rows_ = np.stack([row_of(queries[offs[i]:offs[i + 1]]) for i in range(lengths.size)])
        self.lens = lengths.tolist()
        FakeSlot.log.append(self.lens)

    def poll(self):
        if not self.gate.event.is_set():
            return False
        if self.fail_poll is not None and self.fail_poll in self.lens:
            raise RuntimeError("search failed")
        return True

    def rows(self, n):
        if self.fail_rows is not None and self.fail_rows in self.lens:
            raise RuntimeError("copy to the host failed")
        return self.rows_[:n]

    def close(self):
        pass


def server(gate, slots=2, max_batch=4, max_batch_residues=100, memory_budget=None, **fail):
    FakeSlot.log = []
    db = types.SimpleNamespace(n=N_SUBJECTS, device=0, residues=1)
    return serve.Server(db, slots=slots, max_batch=max_batch,
                        max_batch_residues=max_batch_residues, memory_budget=memory_budget,
                        slot_factory=lambda *a: FakeSlot(gate, **fail))


def queries(sizes, seed=0):
    rng = np.random.default_rng(seed)
    return [rng.integers(0, 20, size=s).astype(np.uint8) for s in sizes]


def test_batches_keep_the_limits_and_the_arrival_order():
    gate = Gate()
    srv = server(gate, slots=2, max_batch=3, max_batch_residues=60)
    qs = queries([10, 25, 5, 30, 30, 1, 2, 3, 59, 60, 20, 20, 20, 20])
    try:
        futs = [srv.submit(q) for q in qs]
        gate.event.set()
        got = [f.result(10) for f in futs]
    finally:
        gate.event.set()
        srv.close(timeout=10)
    for q, g in zip(qs, got):
        assert (g == row_of(q)).all()                       # each request its own row
    rep = srv.report()
    assert rep["requests"] == len(qs) and rep["batches"] == len(FakeSlot.log)
    assert rep["batches"] < len(qs)                         # requests were batched
    for lens in FakeSlot.log:
        assert 1 <= len(lens) <= 3 and sum(lens) <= 60
    # batches take the queue in order: their sizes, concatenated, are the submissions
    assert [s for lens in FakeSlot.log for s in lens] == [q.size for q in qs]
    by_batch = {}
    for r in srv.completed:
        by_batch.setdefault(r.batch, []).append(r.rid)
    ids = [rid for b in sorted(by_batch) for rid in sorted(by_batch[b])]
    assert ids == list(range(len(qs)))
    assert all(r.arrival <= r.admitted <= r.started <= r.finished for r in srv.completed)


def test_batches_overlap_on_free_slots():
    gate = Gate()
    srv = server(gate, slots=3, max_batch=1)
    try:
        futs = [srv.submit(q) for q in queries([5, 6, 7, 8])]
        deadline = time.time() + 10
        while len(FakeSlot.log) < 3 and time.time() < deadline:
            time.sleep(0.001)
        time.sleep(0.01)
        assert len(FakeSlot.log) == 3               # three slots busy, the fourth waits
        gate.event.set()
        [f.result(10) for f in futs]
    finally:
        gate.event.set()
        srv.close(timeout=10)
    assert srv.max_concurrent == 3 and len(FakeSlot.log) == 4


def test_memory_budget_holds_requests_until_rows_are_freed():
    gate = Gate()
    probe = server(Gate(True), slots=1)
    per = probe.request_bytes(10)
    probe.close()
    srv = server(gate, slots=4, max_batch=1, memory_budget=2 * per)
    try:
        futs = [srv.submit(q) for q in queries([10, 10, 10, 10])]
        deadline = time.time() + 10
        while len(FakeSlot.log) < 2 and time.time() < deadline:
            time.sleep(0.001)
        time.sleep(0.01)
        assert len(FakeSlot.log) == 2 and srv._in_use == 2 * per   # two fit the budget
        gate.event.set()
        [f.result(10) for f in futs]
    finally:
        gate.event.set()
        srv.close(timeout=10)
    assert len(FakeSlot.log) == 4 and srv._in_use == 0
    small = server(gate, memory_budget=per - 1)
    try:
        with pytest.raises(serve.AdmissionError):
            small.submit(queries([10])[0])
    finally:
        small.close(timeout=10)


def test_the_default_budget_admits_every_slot_full():
    gate = Gate()
    srv = server(gate, slots=2, max_batch=3, max_batch_residues=30)
    try:
        with srv._lock:     # all seven queued before the scheduler looks (the lock is reentrant)
            futs = [srv.submit(q) for q in queries([10] * 7)]
        deadline = time.time() + 10
        while sum(len(b) for b in FakeSlot.log) < 6 and time.time() < deadline:
            time.sleep(0.001)
        assert [len(b) for b in FakeSlot.log] == [3, 3]    # both slots full; one waits
        gate.event.set()
        [f.result(10) for f in futs]
    finally:
        gate.event.set()
        srv.close(timeout=10)


def test_a_failed_search_fails_only_its_own_batch():
    gate = Gate(True)
    srv = server(gate, slots=1, max_batch=1, fail_poll=13)
    try:
        futs = [srv.submit(q) for q in queries([4, 13, 5])]
        with pytest.raises(RuntimeError, match="search failed"):
            futs[1].result(10)
        assert (futs[0].result(10) == row_of(queries([4])[0])).all()
        assert (futs[2].result(10) == row_of(queries([4, 13, 5])[2])).all()
    finally:
        srv.close()
    assert srv._in_use == 0


def test_a_failed_copy_of_the_rows_fails_only_its_own_batch():
    gate = Gate(True)
    srv = server(gate, slots=1, max_batch=1, fail_rows=13)
    try:
        futs = [srv.submit(q) for q in queries([4, 13, 5])]
        with pytest.raises(RuntimeError, match="copy to the host failed"):
            futs[1].result(10)
        assert (futs[0].result(10) == row_of(queries([4])[0])).all()
        assert (futs[2].result(10) == row_of(queries([4, 13, 5])[2])).all()
        # the scheduler thread is still alive and serving
        assert srv.submit(queries([6])[0]).result(10).shape == (N_SUBJECTS,)
    finally:
        srv.close(timeout=10)
    assert srv._in_use == 0 and not any(s.busy for s in srv.slots)


def test_the_default_budget_stays_within_free_device_memory():
    db = types.SimpleNamespace(n=N_SUBJECTS, device=0, residues=1)
    FakeSlot.log = []
    mk = lambda *a: FakeSlot(Gate(True))  # noqa: E731
    roomy = serve.Server(db, slots=2, max_batch=3, max_batch_residues=30, slot_factory=mk,
                         free_bytes=lambda: 10 ** 9)
    tight = serve.Server(db, slots=2, max_batch=3, max_batch_residues=30, slot_factory=mk,
                         free_bytes=lambda: 100)
    try:
        assert roomy.memory_budget == 2 * (3 * roomy.request_bytes(0) + 30)   # the slots full
        assert tight.memory_budget == 90                                    # 90% of what is free
        assert tight.free_at_start == 100
        # two requests fit 90 bytes (4 x 7 + 10 each), a third waits for one to finish
        per = tight.request_bytes(10)
        assert 2 * per <= 90 < 3 * per
        futs = [tight.submit(q) for q in queries([10] * 5)]
        [f.result(10) for f in futs]
        assert tight.max_in_use <= 90
    finally:
        roomy.close(timeout=10)
        tight.close(timeout=10)


def test_a_failed_launch_fails_only_its_own_batch():
    gate = Gate(True)
    srv = server(gate, slots=2, max_batch=1, fail_launch=9)
    try:
        futs = [srv.submit(q) for q in queries([9, 3])]
        with pytest.raises(RuntimeError, match="launch failed"):
            futs[0].result(10)
        assert futs[1].result(10).shape == (N_SUBJECTS,)
        assert srv.submit(queries([2])[0]).result(10).shape == (N_SUBJECTS,)
    finally:
        srv.close()
    assert srv._in_use == 0 and not any(s.busy for s in srv.slots)


def test_close_drains_admitted_requests_and_then_refuses():
    gate = Gate()
    srv = server(gate, slots=1, max_batch=2)
    futs = [srv.submit(q) for q in queries([3, 4, 5, 6, 7])]
    threading.Timer(0.05, gate.event.set).start()
    srv.close(timeout=10)
    assert all(f.done() and f.exception() is None for f in futs)
    assert srv.report()["requests"] == 5
    with pytest.raises(RuntimeError, match="closed"):
        srv.submit(queries([3])[0])


def test_refusals_at_submit():
    srv = server(Gate(True), max_batch_residues=50)
    try:
        with pytest.raises(serve.AdmissionError):
            srv.submit(np.zeros(51, np.uint8))              # longer than a batch holds
        with pytest.raises(ValueError):
            srv.submit(np.array([1, 24], np.uint8))         # not a residue code
    finally:
        srv.close()


def test_replay_submits_a_trace_in_time_order():
    from paper_2309_09609_gb300 import synth
    trace = synth.serving_trace(seed=5, n=30, rate=5000.0)
    srv = server(Gate(True), slots=2, max_batch=8, max_batch_residues=100000)
    try:
        futs = serve.replay(srv, trace, timeout=10)
    finally:
        srv.close()
    for i, f in enumerate(futs):
        assert (f.result() == row_of(trace.queries.seq(i))).all()
    arr = sorted(srv.completed, key=lambda r: r.rid)
    assert all(a.arrival <= b.arrival for a, b in zip(arr, arr[1:]))
    rep = srv.report()
    assert rep["requests"] == 30 and rep["p50_ms"] <= rep["p99_ms"]


def test_cancelled_requests_are_dropped_before_launch_and_running_ones_finish():
    gate = Gate()
    srv = server(gate, slots=1, max_batch=1)
    try:
        futs = [srv.submit(q) for q in queries([11, 12, 13, 14])]
        deadline = time.time() + 10
        while not FakeSlot.log and time.time() < deadline:
            time.sleep(0.001)
        assert FakeSlot.log == [[11]]
        assert futs[0].cancel() is False            # launched: running, not cancellable
        assert futs[2].cancel() is True             # still queued
        gate.event.set()
        assert futs[0].result(10).shape == (N_SUBJECTS,)
        assert futs[1].result(10).shape == (N_SUBJECTS,)
        assert futs[3].result(10).shape == (N_SUBJECTS,)
        assert futs[2].cancelled()
    finally:
        gate.event.set()
        srv.close(timeout=10)
    assert [lens for lens in FakeSlot.log] == [[11], [12], [14]]   # 13 never searched
    rep = srv.report()
    assert rep["cancelled"] == 1 and rep["requests"] == 3 and srv._in_use == 0
