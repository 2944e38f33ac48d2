"""CPU oracle for exact Smith-Waterman/Gotoh local alignment scores.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2309_09609_gb300``) never imports it, and the two share no code: the
oracle has its own alphabet, encoder, BLOSUM62 table and gap-convention mapping.

What it follows (arxiv 2309.09609):
  * Section II-B, Eq. 1-3: the H/E/F recurrences, zero H on row and column 0,
    score = the largest H (scalar int32 C in ``sw_oracle.c``).
  * Section IV-A: BLOSUM62 scoring, gap penalties "10/2".

Readings of the paper taken here, where it is silent or open to two readings:
  * Gap convention: the library's ``(gap_open, gap_extend)`` means a gap of k
    residues costs ``gap_open + k * gap_extend``.  In the notation of Eq. 2-3
    that is ``Go = gap_open + gap_extend`` and ``Ge = gap_extend``.  The
    paper-literal ``(Go, Ge)`` form is available as ``sw_score_paper``.
  * E and F start at minus infinity on the borders; the paper's zero start is
    ``sw_score_paper(..., zero_init=True)``; both give the same score for
    non-negative penalties (a test checks this).
  * Alphabet: the 24 BLOSUM62 symbols ARNDCQEGHILKMFPSTWYVBZX*; U, O, J and any
    other letter encode as X.

Pins (tests/test_oracle_pins.py): brute-force enumeration of every local
alignment on sequences of length <= 6, the ungapped closed form (Kadane over
diagonals) for huge gap penalties, the textbook linear-gap Smith-Waterman for
Go == Ge, the longest common substring (difflib) for an identity matrix,
score invariants, and BLOSUM62's published Karlin-Altschul lambda and H.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRCS = [os.path.join(_HERE, f) for f in ("sw_oracle.c", "sw_align_oracle.c")]

ALPHABET = "ARNDCQEGHILKMFPSTWYVBZX*"
CODE_X = ALPHABET.index("X")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C files with gcc -O2 (scalar: tree vectorisation off)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = not os.path.exists(_SO) or any(os.path.getmtime(_SO) < os.path.getmtime(f) for f in _SRCS)
    if force or stale:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-fno-tree-vectorize", "-fPIC", "-shared", "-std=c99",
            "-Wall", "-o", tmp] + _SRCS + ["-lpthread"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            for name in ("oracle_sw_gotoh", "oracle_sw_gotoh_zero_init"):
                f = getattr(lib, name)
                f.restype = i32
                f.argtypes = [P, i32, P, i32, P, i32, i32, i32]
            lib.oracle_pairs.restype = i32
            lib.oracle_pairs.argtypes = [P, P, P, P, P, P, P, P, i64, P, i32, i32, i32, P, i32]
            lib.oracle_sw_align.restype = i32
            lib.oracle_sw_align.argtypes = [P, i32, P, i32, P, i32, i32, i32, P, P, P, P, P, i64, P]
            lib.oracle_blosum62.restype = None
            lib.oracle_blosum62.argtypes = [P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def encode(text: str) -> np.ndarray:
    """One code per character: letters -> codes 0..23 in ALPHABET order (a-z
    folded to A-Z, nothing else), anything else -> X."""
    table = {c: i for i, c in enumerate(ALPHABET)}
    fold = {chr(c): chr(c - 32) for c in range(ord("a"), ord("z") + 1)}
    return np.array([table.get(fold.get(c, c), CODE_X) for c in text], dtype=np.uint8)


def blosum62() -> np.ndarray:
    """The oracle's own BLOSUM62, int32 24 x 24 (order ALPHABET)."""
    out = np.zeros(24 * 24, dtype=np.int8)
    _load().oracle_blosum62(_ptr(out))
    return out.reshape(24, 24).astype(np.int32)


def paper_gaps(gap_open: int, gap_extend: int) -> tuple[int, int]:
    """Library convention -> (Go, Ge) of Eq. 2-3 (cost(k) = open + k*extend)."""
    return int(gap_open) + int(gap_extend), int(gap_extend)


def _matrix(matrix) -> np.ndarray:
    sm = blosum62() if matrix is None else np.asarray(matrix)
    sm = np.ascontiguousarray(sm, dtype=np.int32)
    assert sm.ndim == 2 and sm.shape[0] == sm.shape[1]
    return sm


def sw_score_paper(q, d, Go: int, Ge: int, matrix=None, zero_init: bool = False) -> int:
    """S for one pair with Eq. 2-3's own Go/Ge (a gap of k costs Go+(k-1)Ge)."""
    q = np.ascontiguousarray(q, dtype=np.uint8)
    d = np.ascontiguousarray(d, dtype=np.uint8)
    sm = _matrix(matrix)
    if q.size and int(q.max()) >= sm.shape[0] or d.size and int(d.max()) >= sm.shape[0]:
        raise ValueError("residue code outside the scoring matrix")
    f = _load().oracle_sw_gotoh_zero_init if zero_init else _load().oracle_sw_gotoh
    s = f(_ptr(q), q.size, _ptr(d), d.size, _ptr(sm), sm.shape[0], int(Go), int(Ge))
    if s < 0:
        raise MemoryError("oracle allocation failed")
    return int(s)


def align_paper(q, d, Go: int, Ge: int, matrix=None) -> dict:
    """The optimal local alignment of one pair (``sw_align_oracle.c``, which
    states which of several optimal alignments is returned), with Eq. 2-3's
    own Go/Ge: score, 0-based half-open ranges q[q_begin:q_end] and
    d[s_begin:s_end], and the transcript ('M', 'I' = query residue against a
    gap, 'D' = subject residue against a gap), first column to last."""
    q = np.ascontiguousarray(q, dtype=np.uint8)
    d = np.ascontiguousarray(d, dtype=np.uint8)
    sm = _matrix(matrix)
    if q.size and int(q.max()) >= sm.shape[0] or d.size and int(d.max()) >= sm.shape[0]:
        raise ValueError("residue code outside the scoring matrix")
    cap = q.size + d.size
    ops = ctypes.create_string_buffer(max(cap, 1))
    b = np.zeros(4, dtype=np.int32)
    n_ops = ctypes.c_int64(0)
    i4 = [ctypes.byref(ctypes.c_int32.from_buffer(b, 4 * k)) for k in range(4)]
    s = _load().oracle_sw_align(_ptr(q), q.size, _ptr(d), d.size, _ptr(sm), sm.shape[0],
                                int(Go), int(Ge), *i4, ops, cap, ctypes.byref(n_ops))
    if s < 0:
        raise MemoryError("oracle allocation failed")
    return {"score": int(s), "q_begin": int(b[0]), "q_end": int(b[1]), "s_begin": int(b[2]),
            "s_end": int(b[3]), "ops": ops.raw[:n_ops.value].decode()}


def align(q, d, gap_open: int = 10, gap_extend: int = 2, matrix=None) -> dict:
    """``align_paper`` in the library's gap convention (cost(k) = open + k*extend)."""
    Go, Ge = paper_gaps(gap_open, gap_extend)
    return align_paper(q, d, Go, Ge, matrix)


def sw_score(q, d, gap_open: int = 10, gap_extend: int = 2, matrix=None) -> int:
    """S for one pair in the library's gap convention (cost(k) = open + k*extend)."""
    Go, Ge = paper_gaps(gap_open, gap_extend)
    return sw_score_paper(q, d, Go, Ge, matrix)


def _concat(seqs):
    seqs = [np.ascontiguousarray(s, dtype=np.uint8) for s in seqs]
    lens = np.array([s.size for s in seqs], dtype=np.int32)
    offs = np.zeros(len(seqs), dtype=np.int64)
    if len(seqs) > 1:
        offs[1:] = np.cumsum(lens[:-1], dtype=np.int64)
    res = np.concatenate(seqs) if seqs and lens.sum() else np.zeros(1, dtype=np.uint8)
    return res, offs, lens


def _threads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


def pairs_packed(qres, qoff, qlen, dres, doff, dlen, pair_q, pair_d,
                 gap_open=10, gap_extend=2, matrix=None, nthreads=None) -> np.ndarray:
    """Scores of listed (query, subject) pairs over concatenated sequences."""
    Go, Ge = paper_gaps(gap_open, gap_extend)
    sm = _matrix(matrix)
    qres = np.ascontiguousarray(qres, dtype=np.uint8)
    dres = np.ascontiguousarray(dres, dtype=np.uint8)
    if qres.size == 0:
        qres = np.zeros(1, dtype=np.uint8)
    if dres.size == 0:
        dres = np.zeros(1, dtype=np.uint8)
    if int(qres.max()) >= sm.shape[0] or int(dres.max()) >= sm.shape[0]:
        raise ValueError("residue code outside the scoring matrix")
    qoff = np.ascontiguousarray(qoff, dtype=np.int64)
    qlen = np.ascontiguousarray(qlen, dtype=np.int32)
    doff = np.ascontiguousarray(doff, dtype=np.int64)
    dlen = np.ascontiguousarray(dlen, dtype=np.int32)
    pq = np.ascontiguousarray(pair_q, dtype=np.int32)
    pd = np.ascontiguousarray(pair_d, dtype=np.int64)
    out = np.zeros(pq.size, dtype=np.int32)
    rc = _load().oracle_pairs(_ptr(qres), _ptr(qoff), _ptr(qlen), _ptr(dres), _ptr(doff),
                              _ptr(dlen), _ptr(pq), _ptr(pd), pq.size, _ptr(sm),
                              sm.shape[0], Go, Ge, _ptr(out), _threads(nthreads))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return out


def pairs(queries, subjects, pair_q, pair_d, gap_open=10, gap_extend=2, matrix=None,
          nthreads=None) -> np.ndarray:
    """Scores of listed pairs; queries/subjects are lists of code arrays."""
    qres, qoff, qlen = _concat(queries)
    dres, doff, dlen = _concat(subjects)
    return pairs_packed(qres, qoff, qlen, dres, doff, dlen, pair_q, pair_d,
                        gap_open, gap_extend, matrix, nthreads)


def search(queries, subjects, gap_open=10, gap_extend=2, matrix=None,
           nthreads=None) -> np.ndarray:
    """All-pairs scores, shape (len(queries), len(subjects))."""
    nq, nd = len(queries), len(subjects)
    pq = np.repeat(np.arange(nq, dtype=np.int32), nd)
    pd = np.tile(np.arange(nd, dtype=np.int64), nq)
    return pairs(queries, subjects, pq, pd, gap_open, gap_extend, matrix,
                 nthreads).reshape(nq, nd)
