"""sw_search_pairs_noalloc, the entry point for callers that cannot let the
library allocate (a host framework owning all device memory, or a service
that must not allocate while serving).  Called through the C ABI with
caller-owned device buffers, twice in a row, it must give exactly the
oracle's scores (Eq. 1-3) and those of sw_search.  Bad inputs -- a negative
length, a residue code of 24, a host buffer -- return SW_EINVAL and leave the
affected entries of the caller's score buffer untouched.  This file is
collected last so that a failure here stops a `-x` run only after every other
test has run."""
import ctypes

import numpy as np
import pytest

from helpers import concat, oracle_all, seqset
from paper_2309_09609_gb300 import build as nvbuild
from paper_2309_09609_gb300 import swgb, synth

pytestmark = pytest.mark.gpu

SENTINEL = -7


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    nvbuild.build()
    return torch, swgb.lib()


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _noalloc(lib, torch, q, db, gap_open, gap_extend, matrix=None, q_lengths=None,
             s_lengths=None, null_residues=False):
    """One call through the C ABI; returns (status, scores as a host array).
    The score buffer starts filled with SENTINEL."""
    qr = None if null_residues else _dev(torch, q.res if q.res.size else np.zeros(1), np.uint8)
    sr = _dev(torch, db.res if db.res.size else np.zeros(1), np.uint8)
    qo, so = _dev(torch, q.offs, np.int64), _dev(torch, db.offs, np.int64)
    ql = _dev(torch, q.lens if q_lengths is None else q_lengths, np.int32)
    sl = _dev(torch, db.lens if s_lengths is None else s_lengths, np.int32)
    out = torch.full((len(q), len(db)), SENTINEL, dtype=torch.int32, device="cuda")
    m = None if matrix is None else np.ascontiguousarray(matrix, dtype=np.int8).reshape(576)
    P = ctypes.c_void_p
    st = lib.sw_search_pairs_noalloc(
        None if qr is None else P(qr.data_ptr()), P(qo.data_ptr()), P(ql.data_ptr()), len(q),
        P(sr.data_ptr()), P(so.data_ptr()), P(sl.data_ptr()), len(db),
        gap_open, gap_extend, None if m is None else m.ctypes.data_as(P), P(out.data_ptr()), None)
    return st, out.cpu().numpy()


def test_noalloc_matches_the_oracle_and_sw_search_on_two_calls_in_a_row(env):
    torch, lib = env
    rng = np.random.default_rng(99)
    db1 = concat(seqset(rng, [0, 1, 7, 4096, 4095]), seqset(rng, rng.integers(1, 1200, 300)))
    q1 = seqset(rng, [0, 1, 33, 256, 257, 700])
    db2 = seqset(rng, rng.integers(0, 2500, 150))
    q2 = seqset(rng, [5, 144, 513])
    m2 = rng.integers(-4, 7, size=(24, 24)).astype(np.int8)
    for q, db, go, ge, m in [(q1, db1, 10, 2, None), (q2, db2, 5, 1, m2)]:
        st, got = _noalloc(lib, torch, q, db, go, ge, m)
        assert st == swgb.SW_OK, swgb.last_error()
        want = oracle_all(q, db, go, ge, m)
        assert (got == want).all()
        assert (got == swgb.Database.from_seqset(db).search(q.res, q.lens, go, ge, m)).all()


def test_noalloc_rejects_subjects_over_the_limit(env):
    torch, lib = env
    rng = np.random.default_rng(7)
    q, db = seqset(rng, [20]), seqset(rng, [10, 4097])
    st, got = _noalloc(lib, torch, q, db, 10, 2)
    assert st == swgb.SW_EINVAL and "4096" in swgb.last_error()
    assert got[0, 1] == SENTINEL                               # the long subject is not scored
    assert got[0, 0] == oracle_all(q, db.subset([0]))[0, 0]    # the other one is
    # the array is cleared per call: a valid call afterwards succeeds
    db = seqset(rng, [10, 20])
    st, got = _noalloc(lib, torch, q, db, 10, 2)
    assert st == swgb.SW_OK
    assert (got == oracle_all(q, db)).all()


def test_noalloc_negative_length_leaves_its_row_untouched(env):
    torch, lib = env
    rng = np.random.default_rng(8)
    q, db = seqset(rng, [30, 0, 50]), seqset(rng, [40, 60, 5])
    lens = q.lens.copy()
    lens[1] = -1
    st, got = _noalloc(lib, torch, q, db, 10, 2, q_lengths=lens)
    assert st == swgb.SW_EINVAL
    assert (got[1] == SENTINEL).all()
    want = oracle_all(q, db)
    assert (got[[0, 2]] == want[[0, 2]]).all()


def test_noalloc_bad_residue_codes_are_refused_per_pair(env):
    torch, lib = env
    rng = np.random.default_rng(9)
    q, db = seqset(rng, [40, 40]), seqset(rng, [30, 30, 30])
    want = oracle_all(q, db)
    q.res[q.offs[1] + 7] = 24      # a query code outside the alphabet
    db.res[db.offs[2] + 3] = 24    # a subject code outside the alphabet
    st, got = _noalloc(lib, torch, q, db, 10, 2)
    assert st == swgb.SW_EINVAL and "code" in swgb.last_error()
    bad = np.zeros(got.shape, bool)
    bad[1, :] = True
    bad[:, 2] = True
    assert (got[bad] == SENTINEL).all()
    assert (got[~bad] == want[~bad]).all()


def test_noalloc_empty_queries_may_pass_no_residue_buffer(env):
    torch, lib = env
    rng = np.random.default_rng(10)
    q = synth.SeqSet(np.zeros(0, np.uint8), np.zeros(3, np.int32))
    db = seqset(rng, [10, 0, 25])
    st, got = _noalloc(lib, torch, q, db, 10, 2, null_residues=True)
    assert st == swgb.SW_OK, swgb.last_error()
    assert (got == 0).all()
    # a positive length with no residue buffer is refused, not read
    st, got = _noalloc(lib, torch, q, db, 10, 2, q_lengths=np.array([0, 4, 0], np.int32),
                       null_residues=True)
    assert st == swgb.SW_EINVAL
    assert (got[1] == SENTINEL).all() and (got[[0, 2]] == 0).all()


def test_noalloc_refuses_host_buffers_before_any_launch(env):
    torch, lib = env
    rng = np.random.default_rng(11)
    q, db = seqset(rng, [12]), seqset(rng, [9, 14])
    d = {k: _dev(torch, v, t) for k, v, t in [
        ("qr", q.res, np.uint8), ("qo", q.offs, np.int64), ("ql", q.lens, np.int32),
        ("sr", db.res, np.uint8), ("so", db.offs, np.int64), ("sl", db.lens, np.int32)]}
    host_scores = np.full((1, 2), SENTINEL, np.int32)
    P = ctypes.c_void_p
    st = lib.sw_search_pairs_noalloc(
        P(d["qr"].data_ptr()), P(d["qo"].data_ptr()), P(d["ql"].data_ptr()), 1,
        P(d["sr"].data_ptr()), P(d["so"].data_ptr()), P(d["sl"].data_ptr()), 2,
        10, 2, None, host_scores.ctypes.data_as(P), None)
    assert st == swgb.SW_EINVAL and "scores" in swgb.last_error()
    assert (host_scores == SENTINEL).all()
    # the wrapper: tensors on the device, scores right after the refusal
    out = torch.full((1, 2), SENTINEL, dtype=torch.int32, device="cuda")
    swgb.search_pairs_noalloc(d["qr"], d["qo"], d["ql"], d["sr"], d["so"], d["sl"], out)
    assert (out.cpu().numpy() == oracle_all(q, db)).all()
