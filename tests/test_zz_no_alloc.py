"""sw_search_pairs_noalloc, the entry point for callers that cannot let the
library allocate (a host framework owning all device memory, or a service
that must not allocate while serving).  Called through the C ABI with
caller-owned device buffers, twice in a row, it must give exactly the scores
of sw_search.  This file is collected last so that a failure here stops a
`-x` run only after every other test has run."""
import ctypes

import numpy as np
import pytest

from helpers import concat, seqset
from paper_2309_09609_gb300 import build as nvbuild
from paper_2309_09609_gb300 import swgb

pytestmark = pytest.mark.gpu


def _device_set(torch, ss):
    res = torch.from_numpy(ss.res if ss.res.size else np.zeros(1, np.uint8)).cuda()
    return res, torch.from_numpy(ss.offs).cuda(), torch.from_numpy(ss.lens).cuda()


def _noalloc(lib, torch, q, db, gap_open, gap_extend, matrix=None):
    qr, qo, ql = _device_set(torch, q)
    sr, so, sl = _device_set(torch, db)
    out = torch.full((len(q), len(db)), -7, dtype=torch.int32, device="cuda")
    m = None if matrix is None else np.ascontiguousarray(matrix, dtype=np.int8).reshape(576)
    P = ctypes.c_void_p
    st = lib.sw_search_pairs_noalloc(
        P(qr.data_ptr()), P(qo.data_ptr()), P(ql.data_ptr()), len(q),
        P(sr.data_ptr()), P(so.data_ptr()), P(sl.data_ptr()), len(db),
        gap_open, gap_extend, None if m is None else m.ctypes.data_as(P), P(out.data_ptr()), None)
    return st, out.cpu().numpy()


def test_noalloc_matches_sw_search_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    nvbuild.build()
    lib = swgb.lib()
    rng = np.random.default_rng(99)
    db1 = concat(seqset(rng, [0, 1, 7, 4096, 4095]), seqset(rng, rng.integers(1, 1200, 300)))
    q1 = seqset(rng, [0, 1, 33, 256, 257, 700])
    db2 = seqset(rng, rng.integers(0, 2500, 150))
    q2 = seqset(rng, [5, 144, 513])
    m2 = rng.integers(-4, 7, size=(24, 24)).astype(np.int8)
    for q, db, go, ge, m in [(q1, db1, 10, 2, None), (q2, db2, 5, 1, m2)]:
        st, got = _noalloc(lib, torch, q, db, go, ge, m)
        assert st == swgb.SW_OK, swgb.last_error()
        want = swgb.Database.from_seqset(db).search(q.res, q.lens, go, ge, m)
        assert (got == want).all()


def test_noalloc_rejects_subjects_over_the_limit():
    torch = pytest.importorskip("torch")
    nvbuild.build()
    lib = swgb.lib()
    rng = np.random.default_rng(7)
    st, _ = _noalloc(lib, torch, seqset(rng, [20]), seqset(rng, [10, 4097]), 10, 2)
    assert st == swgb.SW_EINVAL and "4096" in swgb.last_error()
    # the array is cleared per call: a valid call afterwards succeeds
    db = seqset(rng, [10, 20])
    q = seqset(rng, [20])
    st, got = _noalloc(lib, torch, q, db, 10, 2)
    assert st == swgb.SW_OK
    assert (got == swgb.Database.from_seqset(db).search(q.res, q.lens)).all()
