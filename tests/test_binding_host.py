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
