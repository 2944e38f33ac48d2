"""The Python binding's argument marshalling, on the CPU: buffers of the wrong
type, size or layout are refused before any library call, so that a caller's
mistake can never make the library read or write past a buffer."""
import numpy as np
import pytest

from paper_2309_09609_gb300 import swgb

torch = pytest.importorskip("torch")


def test_scores_out_is_checked():
    a = swgb._scores_out(None, 3, 5)
    assert a.shape == (3, 5) and a.dtype == np.int32
    ok = np.zeros((3, 5), np.int32)
    assert swgb._scores_out(ok, 3, 5) is ok
    assert swgb._scores_out(np.zeros(15, np.int32), 3, 5).size == 15     # any shape of that size
    for bad in [np.zeros((3, 4), np.int32),                  # too small: would be overrun
                np.zeros((3, 5), np.int64),                  # wrong element type
                np.zeros((5, 3), np.int32).T,                # not C-contiguous
                [[0] * 5] * 3]:                              # not an array
        with pytest.raises(ValueError):
            swgb._scores_out(bad, 3, 5)
    ro = np.zeros((3, 5), np.int32)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        swgb._scores_out(ro, 3, 5)
    t = torch.zeros((3, 5), dtype=torch.int32)
    assert swgb._scores_out(t, 3, 5) is t
    for bad in [torch.zeros((3, 5), dtype=torch.int64), torch.zeros((2, 5), dtype=torch.int32),
                torch.zeros((5, 3), dtype=torch.int32).t()]:
        with pytest.raises(ValueError):
            swgb._scores_out(bad, 3, 5)


def test_matrix_is_checked():
    m = swgb._matrix(np.arange(576).reshape(24, 24) % 11 - 5)
    assert m.dtype == np.int8 and m.shape == (576,) and m[7] == 2
    assert swgb._matrix(None) is None
    with pytest.raises(ValueError):
        swgb._matrix(np.zeros((20, 20)))
    with pytest.raises(ValueError):
        swgb._matrix(np.full((24, 24), 200))
    with pytest.raises(TypeError):
        swgb._matrix(torch.zeros((24, 24), dtype=torch.int32))
    assert swgb._matrix(torch.zeros((24, 24), dtype=torch.int8)).is_contiguous()


def test_element_types_are_converted():
    x = swgb._as(torch.tensor([1, 2, 3], dtype=torch.int64), "int32")
    assert x.dtype == torch.int32 and x.tolist() == [1, 2, 3]
    y = swgb._as([5, 6], "uint8")
    assert isinstance(y, np.ndarray) and y.dtype == np.uint8
    h = swgb._host(torch.tensor([[1, 2], [3, 4]], dtype=torch.int16), "int64")
    assert isinstance(h, np.ndarray) and h.dtype == np.int64 and h.tolist() == [[1, 2], [3, 4]]


def test_pointers_need_contiguous_buffers():
    with pytest.raises(ValueError):
        swgb._ptr(np.zeros((4, 4), np.int32)[:, 1])
    with pytest.raises(ValueError):
        swgb._ptr(torch.zeros((4, 4))[:, 1])
    with pytest.raises(ValueError):
        swgb._ptr([1, 2, 3])
    assert swgb._ptr(None) is None
    a = np.zeros(4, np.int32)
    assert swgb._ptr(a).value == a.ctypes.data


def test_noalloc_wants_gpu_tensors_of_the_stated_types():
    q = torch.zeros(4, dtype=torch.uint8)
    off = torch.zeros(1, dtype=torch.int64)
    ln = torch.full((1,), 4, dtype=torch.int32)
    sc = torch.zeros((1, 1), dtype=torch.int32)
    with pytest.raises(TypeError, match="queries must be a uint8 torch tensor on the GPU"):
        swgb.search_pairs_noalloc(q, off, ln, q, off, ln, sc)       # host tensors
    with pytest.raises(TypeError, match="queries"):
        swgb.search_pairs_noalloc(q.numpy(), off, ln, q, off, ln, sc)   # numpy


class FakeCudaTensor:
    """Stands in for a CUDA tensor on a given device (no GPU here): only the
    attributes the binding's checks read."""

    def __init__(self, dtype, n, index):
        self.dtype, self.shape, self.is_cuda = dtype, (n,), True
        self.device = type("Dev", (), {"index": index})()

    def data_ptr(self):
        return 0

    def numel(self):
        return self.shape[0]

    def is_contiguous(self):
        return True


def test_noalloc_wants_every_tensor_on_one_device():
    args = [FakeCudaTensor("torch.uint8", 4, 0), FakeCudaTensor("torch.int64", 1, 0),
            FakeCudaTensor("torch.int32", 1, 0), FakeCudaTensor("torch.uint8", 4, 1),
            FakeCudaTensor("torch.int64", 1, 0), FakeCudaTensor("torch.int32", 1, 0),
            FakeCudaTensor("torch.int32", 1, 0)]
    with pytest.raises(ValueError, match=r"one GPU, got devices \[0, 1\]"):
        swgb.search_pairs_noalloc(*args)


class FakeLib:
    """Stands in for libswgb.so: records every call, returns SW_OK.  Handles
    it creates stay NULL, so closing them is a no-op with any library."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append((name, args))
            return 0
        return call

    def last(self, name):
        return [a for n, a in self.calls if n == name][-1]


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib()
    f.sw_last_error = lambda: b""
    monkeypatch.setattr(swgb, "_lib", f)
    return f


def test_wrappers_pass_counts_and_buffers_of_the_stated_types(fake):
    db = swgb.Database(np.array([1, 2, 3, 4, 5], np.uint8), [2, 3])
    assert db.n == 2 and db.subject_lengths().tolist() == [2, 3]
    res, lens, n, dev, _ = fake.last("sw_db_create")
    assert n == 2 and dev == 0
    out = db.search([4, 5, 6], torch.tensor([1, 2], dtype=torch.int64), 10, 2)
    assert out.shape == (2, 2) and out.dtype == np.int32
    h, q, ql, nq, go, ge, m, sc, st = fake.last("sw_search")
    assert nq == 2 and (go, ge) == (10, 2) and m is None and st is None
    plan = db.plan(4, 100, rows_per_thread=16)
    o = fake.last("sw_plan_create")[3]._obj
    assert o.rows_per_thread == 16
    buf = np.zeros((1, 2), np.int32)
    assert plan.search(np.array([7], np.uint8), [1], out=buf) is buf
    with pytest.raises(ValueError):
        plan.search(np.array([7], np.uint8), [1], out=np.zeros((2, 2), np.int32))
    dev_out = torch.zeros((1, 2), dtype=torch.int32)
    plan.search_async(torch.tensor([7], dtype=torch.uint8), [1], dev_out)
    assert fake.last("sw_plan_search_async")[3] == 1
    assert plan.wait(0) is True and isinstance(plan.stats(), dict)


def test_align_sizes_the_transcript_buffer_and_checks_indices(fake):
    db = swgb.Database(np.arange(10, dtype=np.uint8) % 20, [4, 6])
    q, ql = np.arange(7, dtype=np.uint8), np.array([3, 4], np.int32)
    got = db.align(q, ql, [0, 1, 1], [1, 0, 1])
    assert len(got) == 3 and all(g["ops"] == "" for g in got)
    args = fake.last("sw_align")
    n_pairs, ops_capacity = args[6], args[12]
    assert n_pairs == 3 and ops_capacity == (3 + 6) + (4 + 4) + (4 + 6)
    for pq, ps in [([2], [0]), ([-1], [0]), ([0], [2]), ([0], [-1])]:
        with pytest.raises(swgb.SwError) as e:
            db.align(q, ql, pq, ps)
        assert e.value.status == swgb.SW_EINVAL
    with pytest.raises(ValueError):
        db.align(q, ql, [0, 1], [0])
    assert db.align(q, ql, [], []) == []


def test_a_failing_call_raises_with_the_library_message(fake, monkeypatch):
    monkeypatch.setattr(fake, "sw_last_error", lambda: b"queries is NULL", raising=False)
    fake.sw_search = lambda *a: swgb.SW_EINVAL
    db = swgb.Database(np.array([1], np.uint8), [1])
    with pytest.raises(swgb.SwError, match="SW_EINVAL: queries is NULL") as e:
        db.search([1], [1])
    assert e.value.status == swgb.SW_EINVAL


def test_a_closed_database_is_refused_by_the_library():
    # the real libswgb: a closed handle is NULL, which every entry point
    # rejects with SW_EINVAL before any CUDA call
    from paper_2309_09609_gb300 import build as nvbuild
    nvbuild.build()
    swgb.lib()
    db = object.__new__(swgb.Database)
    db._h, db.n, db.device, db._lens = None, 2, 0, np.array([3, 4], np.int32)
    for call in (lambda: db.search([1, 2], [2]),
                 lambda: db.search_plain([1, 2], [2]),
                 lambda: db.plan(1, 2),
                 lambda: db.align(np.array([1, 2], np.uint8), [2], [0], [1])):
        with pytest.raises(swgb.SwError) as e:
            call()
        assert e.value.status == swgb.SW_EINVAL and "NULL" in str(e.value)


def test_top_hits_orders_by_score_then_subject():
    s = np.array([[5, 9, 9, 0, 7], [0, 0, 0, 0, 0], [1, 2, 3, 4, 5]], np.int32)
    idx, val = swgb.top_hits(s, 3)
    assert idx.tolist() == [[1, 2, 4], [0, 1, 2], [4, 3, 2]]
    assert val.tolist() == [[9, 9, 7], [0, 0, 0], [5, 4, 3]]
    idx, val = swgb.top_hits(torch.from_numpy(s), 10)      # k larger than the subjects
    assert idx.shape == (3, 5) and val[0].tolist() == [9, 9, 7, 5, 0]
    assert swgb.top_hits(s, 0)[0].shape == (3, 0)
    with pytest.raises(ValueError):
        swgb.top_hits(s[0], 2)
