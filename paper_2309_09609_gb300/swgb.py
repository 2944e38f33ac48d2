"""Thin ctypes binding of libswgb (include/swgb.h): argument marshalling only.

Every step of a search runs in the library's CUDA kernels.  There is no CPU
fallback: if ``_build/libswgb.so`` is missing, loading raises.  Arrays may be
numpy arrays (host) or torch tensors (host or CUDA); a torch stream or a raw
``cudaStream_t`` integer selects the stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libswgb.so")

SW_OK, SW_EINVAL, SW_ENOMEM, SW_ECUDA, SW_ETIMEDOUT, SW_EBUSY = range(6)
_STATUS = {1: "SW_EINVAL", 2: "SW_ENOMEM", 3: "SW_ECUDA", 4: "SW_ETIMEDOUT", 5: "SW_EBUSY"}
ALPHABET = "ARNDCQEGHILKMFPSTWYVBZX*"

#: intpeak op codes (sw_intpeak)
INTPEAK_OPS = ["iadd", "imax", "viaddmax_s32", "viaddmax_s16x2", "viaddmax_s16x2_relu",
               "vimax3_s16x2", "vmaxs2", "vsub2", "vaddss2", "prmt", "cell_s16x2",
               "cell_s16x2_prmt", "cell_i32", "imad", "cell_biased", "vadd4", "vmaxu4",
               "vmaxs4", "vaddus4", "vsubus4", "cell_u8x4"]


class SwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("rows_per_thread", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("long_cutoff", ctypes.c_int32), ("intra_rows", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("force_int32", ctypes.c_int32),
                ("auto_cutoff", ctypes.c_int32), ("wide_min_len", ctypes.c_int32),
                ("wide_min_subject", ctypes.c_int32), ("inter_columns", ctypes.c_int32),
                ("overlap_kernels", ctypes.c_int32), ("two_query", ctypes.c_int32),
                ("two_query_rows", ctypes.c_int32), ("two_query_pairs", ctypes.c_int32),
                ("flag_capacity", ctypes.c_int32), ("two_query_long", ctypes.c_int32)]


class Alignment(ctypes.Structure):
    _fields_ = [("score", ctypes.c_int32), ("q_begin", ctypes.c_int32), ("q_end", ctypes.c_int32),
                ("s_begin", ctypes.c_int32), ("s_end", ctypes.c_int32), ("n_ops", ctypes.c_int32),
                ("ops_offset", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_int64), ("inter_items", ctypes.c_int64),
                ("intra_items", ctypes.c_int64), ("recomputed_pairs", ctypes.c_int64),
                ("overflow_rounds", ctypes.c_int32), ("kernels_launched", ctypes.c_int32),
                ("search_ms", ctypes.c_float), ("recompute_ms", ctypes.c_float),
                ("pair_ms", ctypes.c_float), ("pad_", ctypes.c_int32),
                ("inter_cells", ctypes.c_int64), ("inter2_items", ctypes.c_int64),
                ("pair2_items", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None


def lib():
    """Loads libswgb.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libswgb.so is missing ({LIB_PATH}); build it with "
                               "`python -m paper_2309_09609_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        sig = {
            "sw_last_error": (ctypes.c_char_p, []),
            "sw_encode": (i32, [P, i64, P]),
            "sw_default_matrix": (None, [P]),
            "sw_db_create": (i32, [P, P, i64, ctypes.c_int, ctypes.POINTER(P)]),
            "sw_db_destroy": (None, [P]),
            "sw_db_subjects": (i64, [P]),
            "sw_db_residues": (i64, [P]),
            "sw_db_max_length": (i32, [P]),
            "sw_options_default": (None, [ctypes.POINTER(Options)]),
            "sw_plan_create": (i32, [P, i32, i64, ctypes.POINTER(Options), ctypes.POINTER(P)]),
            "sw_plan_destroy": (None, [P]),
            "sw_plan_search": (i32, [P, P, P, i32, i32, i32, P, P, P]),
            "sw_plan_search_async": (i32, [P, P, P, i32, i32, i32, P, P, P]),
            "sw_plan_wait": (i32, [P, i32]),
            "sw_plan_stats": (i32, [P, ctypes.POINTER(Stats)]),
            "sw_search": (i32, [P, P, P, i32, i32, i32, P, P, P]),
            "sw_search_plain": (i32, [P, P, P, i32, i32, i32, P, P, P]),
            "sw_intpeak": (i32, [i32, i32, i32, i32, P]),
            "sw_search_pairs_noalloc": (i32, [P, P, P, i32, P, P, P, i32, i32, i32, P, P, P]),
            "sw_align": (i32, [P, P, P, i32, P, P, i32, i32, i32, P, P, P, i64, P]),
            "sw_query_streams": (i32, [P, i32, i32, i32, P, i64, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _check(status: int):
    if status != SW_OK:
        raise SwError(status, lib().sw_last_error().decode(errors="replace"))


def last_error() -> str:
    return lib().sw_last_error().decode(errors="replace")


def _ptr(x):
    """Raw pointer of a numpy array or torch tensor (kept alive by the caller)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if not (isinstance(x, np.ndarray) and x.flags.c_contiguous):
        raise ValueError("need a contiguous numpy array")
    return ctypes.c_void_p(x.ctypes.data)


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _as(x, dtype: str):
    """x as a contiguous array of `dtype` ("uint8", "int8", "int32", "int64"):
    numpy input becomes a numpy array, a torch tensor stays a tensor on its
    own device (converted there when its dtype differs)."""
    if hasattr(x, "data_ptr"):
        if str(x.dtype) != "torch." + dtype:
            x = x.to(getattr(__import__("torch"), dtype))
        return x.contiguous()
    return np.ascontiguousarray(x, dtype=getattr(np, dtype))


def _host(x, dtype: str) -> np.ndarray:
    """x as a contiguous host numpy array of `dtype` (torch tensors are copied
    to the host), for arguments the library reads on the host."""
    if hasattr(x, "data_ptr"):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(x, dtype=getattr(np, dtype))


def _u8(x):
    return _as(x, "uint8")


def _i32(x):
    return _as(x, "int32")


def _matrix(m):
    """A 24 x 24 substitution matrix as 576 int8 (NULL, i.e. BLOSUM62, for None)."""
    if m is None:
        return None
    if hasattr(m, "data_ptr"):
        if m.numel() != 576:
            raise ValueError("matrix must be 24 x 24")
        if str(m.dtype) != "torch.int8":
            raise TypeError("a matrix tensor must be int8")
        return m.contiguous()
    m = np.ascontiguousarray(m)
    if m.size != 576:
        raise ValueError("matrix must be 24 x 24")
    if m.min() < -128 or m.max() > 127:
        raise ValueError("matrix entries must fit int8")
    return np.ascontiguousarray(m.astype(np.int8).reshape(576))


def _scores_out(out, nq: int, ns: int):
    """The caller's score buffer (int32, nq x ns, contiguous), or a new host
    array when out is None."""
    if out is None:
        return np.empty((nq, ns), dtype=np.int32)
    if hasattr(out, "data_ptr"):
        ok = str(out.dtype) == "torch.int32" and out.numel() == nq * ns and out.is_contiguous()
    else:
        ok = (isinstance(out, np.ndarray) and out.dtype == np.int32 and out.size == nq * ns
              and out.flags.c_contiguous and out.flags.writeable)
    if not ok:
        raise ValueError(f"out must be a contiguous, writable int32 buffer of {nq} x {ns}")
    return out


def encode(text: str) -> np.ndarray:
    b = text.encode("latin-1")
    out = np.empty(len(b), dtype=np.uint8)
    src = np.frombuffer(b, dtype=np.uint8) if b else np.zeros(1, np.uint8)
    _check(lib().sw_encode(_ptr(src), len(b), _ptr(out) if len(b) else None))
    return out


def default_matrix() -> np.ndarray:
    out = np.zeros(576, dtype=np.int8)
    lib().sw_default_matrix(_ptr(out))
    return out.reshape(24, 24)


def options(**kw) -> Options:
    o = Options()
    lib().sw_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, int(v))
    return o


def _query_args(queries, q_lengths):
    q = _u8(queries)
    ql = _i32(q_lengths)
    n = int(ql.shape[0]) if hasattr(ql, "shape") else len(ql)
    if (hasattr(q, "numel") and q.numel() == 0) or (isinstance(q, np.ndarray) and q.size == 0):
        q = np.zeros(1, np.uint8)
    return q, ql, n


class Database:
    """A protein database resident on one GPU (sw_db_create)."""

    def __init__(self, residues, lengths, device: int = 0):
        # sw_db_create reads both arrays on the host
        res = _host(residues, "uint8").reshape(-1)
        lens = _host(lengths, "int32").reshape(-1)
        n = int(lens.shape[0])
        if res.size == 0:
            res = np.zeros(1, np.uint8)
        h = ctypes.c_void_p()
        _check(lib().sw_db_create(_ptr(res), _ptr(lens) if n else None, n, device, ctypes.byref(h)))
        self._h = h
        self.device = device
        self.n = n
        self._lens = lens.copy()

    def subject_lengths(self) -> np.ndarray:
        """Subject lengths in caller order (host copy)."""
        return self._lens

    @classmethod
    def from_seqset(cls, ss, device: int = 0):
        return cls(ss.res, ss.lens, device)

    def close(self):
        if getattr(self, "_h", None):
            lib().sw_db_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def residues(self) -> int:
        return int(lib().sw_db_residues(self._h))

    @property
    def max_length(self) -> int:
        return int(lib().sw_db_max_length(self._h))

    def _out(self, nq, out):
        return _scores_out(out, nq, self.n)

    def search(self, queries, q_lengths, gap_open=10, gap_extend=2, matrix=None, out=None,
               stream=None):
        """One-shot exact search (sw_search); returns scores [nq, n_subjects]."""
        q, ql, nq = _query_args(queries, q_lengths)
        out = self._out(nq, out)
        m = _matrix(matrix)
        _check(lib().sw_search(self._h, _ptr(q), _ptr(ql), nq, gap_open, gap_extend, _ptr(m),
                               _ptr(out), _stream(stream)))
        return out

    def search_plain(self, queries, q_lengths, gap_open=10, gap_extend=2, matrix=None, out=None,
                     stream=None):
        """The int32 one-query-per-launch baseline (sw_search_plain)."""
        q, ql, nq = _query_args(queries, q_lengths)
        out = self._out(nq, out)
        m = _matrix(matrix)
        _check(lib().sw_search_plain(self._h, _ptr(q), _ptr(ql), nq, gap_open, gap_extend,
                                     _ptr(m), _ptr(out), _stream(stream)))
        return out

    def align(self, queries, q_lengths, pair_query, pair_subject, gap_open=10, gap_extend=2,
              matrix=None, stream=None) -> list[dict]:
        """Optimal local alignments with traceback of the given (query index,
        subject index) pairs (sw_align): per pair the score, 0-based
        half-open ranges q[q_begin:q_end] and s[s_begin:s_end], and the
        transcript ('M', 'I' = query residue against a gap, 'D' = subject
        residue against a gap), first column to last."""
        q, ql, nq = _query_args(queries, q_lengths)
        pq = _host(pair_query, "int32")
        ps = _host(pair_subject, "int64")
        if pq.ndim != 1 or pq.shape != ps.shape:
            raise ValueError("pair_query and pair_subject must be 1-D and of one length")
        lens = _host(ql, "int32")
        if pq.size and (pq.min() < 0 or pq.max() >= nq):
            raise SwError(SW_EINVAL, "pair_query out of range")
        if ps.size and (ps.min() < 0 or ps.max() >= self.n):
            raise SwError(SW_EINVAL, "pair_subject out of range")
        need = int(sum(int(lens[a]) for a in pq)) + int(self.subject_lengths()[ps].sum()) \
            if pq.size else 0
        ops = np.zeros(max(need, 1), dtype=np.uint8)
        out = (Alignment * max(pq.size, 1))()
        m = _matrix(matrix)
        _check(lib().sw_align(self._h, _ptr(q), _ptr(ql), nq, _ptr(pq), _ptr(ps), pq.size,
                              gap_open, gap_extend, _ptr(m), out, _ptr(ops), ops.size,
                              _stream(stream)))
        res = []
        for k in range(pq.size):
            r = out[k]
            res.append({"score": r.score, "q_begin": r.q_begin, "q_end": r.q_end,
                        "s_begin": r.s_begin, "s_end": r.s_end,
                        "ops": ops[r.ops_offset:r.ops_offset + r.n_ops].tobytes().decode()})
        return res

    def plan(self, max_queries: int, max_query_residues: int, **opts) -> "Plan":
        return Plan(self, max_queries, max_query_residues, options(**opts))


class Plan:
    """A reusable search context (sw_plan_create): buffers + CUDA graph."""

    def __init__(self, db: Database, max_queries: int, max_query_residues: int, opts=None):
        h = ctypes.c_void_p()
        _check(lib().sw_plan_create(db._h, int(max_queries), int(max_query_residues),
                                    ctypes.byref(opts) if opts is not None else None,
                                    ctypes.byref(h)))
        self._h = h
        self.db = db
        self.max_queries = int(max_queries)
        self.max_query_residues = int(max_query_residues)
        self._keep = None

    def close(self):
        if getattr(self, "_h", None):
            lib().sw_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def search(self, queries, q_lengths, gap_open=10, gap_extend=2, matrix=None, out=None,
               stream=None):
        q, ql, nq = _query_args(queries, q_lengths)
        out = _scores_out(out, nq, self.db.n)
        m = _matrix(matrix)
        _check(lib().sw_plan_search(self._h, _ptr(q), _ptr(ql), nq, gap_open, gap_extend,
                                    _ptr(m), _ptr(out), _stream(stream)))
        return out

    def search_async(self, queries, q_lengths, out, gap_open=10, gap_extend=2, matrix=None,
                     stream=None):
        """Queues a search; `out` must be device memory (e.g. a CUDA tensor).
        The queries and lengths are read on the host before this returns."""
        q, ql, nq = _query_args(_host(queries, "uint8"), _host(q_lengths, "int32"))
        out = _scores_out(out, nq, self.db.n)
        m = _matrix(matrix)
        self._keep = (q, ql, m, out)
        _check(lib().sw_plan_search_async(self._h, _ptr(q), _ptr(ql), nq, gap_open, gap_extend,
                                          _ptr(m), _ptr(out), _stream(stream)))

    def wait(self, timeout_ms: int = -1) -> bool:
        """True when done; False if still running after timeout_ms."""
        st = lib().sw_plan_wait(self._h, int(timeout_ms))
        if st == SW_ETIMEDOUT:
            return False
        _check(st)
        self._keep = None
        return True

    def stats(self) -> dict:
        s = Stats()
        _check(lib().sw_plan_stats(self._h, ctypes.byref(s)))
        return s.as_dict()


def top_hits(scores, k: int):
    """Each query's k best subjects from a score matrix [queries, subjects]
    (numpy or torch, host or device): (subject indices, scores), both
    [queries, min(k, subjects)], best first, ties in subject order.  The
    indices feed ``Database.align`` directly, e.g. with
    ``np.repeat(np.arange(nq), k)`` and ``idx.ravel()``."""
    s = scores.cpu().numpy() if hasattr(scores, "cpu") else np.asarray(scores)
    if s.ndim != 2:
        raise ValueError("scores must be [queries, subjects]")
    k = max(0, min(int(k), s.shape[1]))
    # a stable sort on the negated scores keeps equal scores in subject order
    idx = np.argsort(-s.astype(np.int64), axis=1, kind="stable")[:, :k]
    return idx.astype(np.int64), np.take_along_axis(s, idx, axis=1)


def search_pairs_noalloc(queries, q_offsets, q_lengths, subjects, s_offsets, s_lengths, scores,
                         gap_open=10, gap_extend=2, matrix=None, stream=None):
    """sw_search_pairs_noalloc: all pairs, for callers that cannot let the
    library allocate.  Every array is caller-owned CUDA memory (torch CUDA
    tensors) except `matrix` (host); subjects are at most 4096 residues."""
    want = {"queries": (queries, "uint8"), "q_offsets": (q_offsets, "int64"),
            "q_lengths": (q_lengths, "int32"), "subjects": (subjects, "uint8"),
            "s_offsets": (s_offsets, "int64"), "s_lengths": (s_lengths, "int32"),
            "scores": (scores, "int32")}
    for name, (x, dtype) in want.items():
        if not (hasattr(x, "data_ptr") and x.is_cuda and str(x.dtype) == "torch." + dtype):
            raise TypeError(f"{name} must be a {dtype} torch tensor on the GPU")
    # the library launches on the current device: every tensor must live on
    # one device, which is made current for the call
    devices = {x.device.index for x, _ in want.values()}
    if len(devices) != 1:
        raise ValueError(f"all tensors must be on one GPU, got devices {sorted(devices)}")
    nq, ns = int(q_lengths.shape[0]), int(s_lengths.shape[0])
    if q_offsets.shape[0] != nq or s_offsets.shape[0] != ns:
        raise ValueError("one offset per sequence")
    scores = _scores_out(scores, nq, ns)
    m = None if matrix is None else _host(_matrix(matrix), "int8")   # host memory
    # an empty residue tensor may have no storage: pass NULL (allowed when
    # every length on that side is 0; the library refuses to read it)
    qp = _ptr(queries) if queries.numel() else None
    sp = _ptr(subjects) if subjects.numel() else None
    import torch
    with torch.cuda.device(devices.pop()):
        _check(lib().sw_search_pairs_noalloc(
            qp, _ptr(q_offsets), _ptr(q_lengths), nq,
            sp, _ptr(s_offsets), _ptr(s_lengths), ns,
            gap_open, gap_extend, _ptr(m), _ptr(scores), _stream(stream)))
    return scores


def intpeak(op, blocks_per_sm: int = 8, threads: int = 256, iters: int = 20000):
    """Integer-pipe microbenchmark: (lane-ops per SM clock, SM MHz, seconds)."""
    code = INTPEAK_OPS.index(op) if isinstance(op, str) else int(op)
    out = np.zeros(3, dtype=np.float64)
    _check(lib().sw_intpeak(code, blocks_per_sm, threads, iters, _ptr(out)))
    return float(out[0]), float(out[1]), float(out[2])


def query_streams(q_lengths, rows: int = 32, n_pairs: int = 1):
    """The query streams of the two-query kernels (sw_query_streams, host
    only): (strips, pairs) -- strips an (n, 4) int32 array (query of half 0,
    first row | 0x80000000 on its last strip, the same for half 1; query -1
    for an empty half), pairs a (n_pairs, 2) array (first strip, strips)."""
    lens = np.ascontiguousarray(np.asarray(q_lengths, dtype=np.int32))
    cap = 2 * (int(lens.clip(min=0).sum()) // 16 + 2 * len(lens)) + 16
    strips = np.zeros((cap, 4), dtype=np.int32)
    pairs = np.zeros((max(int(n_pairs), 1), 2), dtype=np.int32)
    n = ctypes.c_int64(0)
    _check(lib().sw_query_streams(_ptr(lens), len(lens), int(rows), int(n_pairs), _ptr(strips),
                                  cap, _ptr(pairs), ctypes.byref(n)))
    return strips[:n.value].copy(), pairs[:int(n_pairs)].copy()
