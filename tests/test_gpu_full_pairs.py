"""Every pair of the full-size workloads against the oracle.

``tests/golden/full_pairs_<name>.txt`` holds, for each query row of a
workload's score matrix, the SHA-256 of the oracle's exact scores against
every subject (Eq. 1-3; written by ``tests/golden/full_pair_digests.py``,
which calls only the oracle).  Each test here redraws the same seeded inputs,
runs the library in the launch configuration the benchmark times, and
compares the digest of every row: one differing score anywhere fails it.  On
a mismatch the oracle rescored a stretch of the row, so that the message
names differing pairs.  Workloads whose digest file has not been written are
skipped.
"""
import importlib.util
import os

import numpy as np
import pytest

import oracle
from paper_2309_09609_gb300 import build as nvbuild
from paper_2309_09609_gb300 import swgb

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location(
    "full_pair_digests", os.path.join(HERE, "golden", "full_pair_digests.py"))
fpd = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(fpd)


@pytest.fixture(scope="module", autouse=True)
def built():
    nvbuild.build()
    swgb.lib()


def golden(name):
    path = fpd.path_of(name)
    if not os.path.exists(path):
        pytest.skip(f"no digest file for {name} (tests/golden/full_pair_digests.py {name})")
    g = fpd.read(path)
    q, db, go, ge, _ = fpd.workload(name)
    assert g["head"]["input_sha256"] == fpd.input_digest(q, db, go, ge), \
        f"{name}: the seeded inputs differ from those the digests were written for"
    assert len(g["rows"]) == len(q)
    return g, q, db, go, ge


def compare_rows(name, g, rows, q, db, go, ge, which=None):
    """rows[k] is the score row of query which[k] (default: k)."""
    which = range(len(rows)) if which is None else which
    bad = []
    for k, i in enumerate(which):
        m, mx, sm, sha = g["rows"][i]
        assert m == int(q.lens[i])
        if fpd.row_digest(rows[k])[2] != sha:
            bad.append((k, i))
    if not bad:
        return
    k, i = bad[0]
    n = min(len(db), 20000)
    pd = np.arange(n, dtype=np.int64)
    want = oracle.pairs_packed(q.res, q.offs, q.lens, db.res, db.offs, db.lens,
                               np.full(n, i, np.int32), pd, go, ge)
    diff = np.nonzero(np.asarray(rows[k][:n]) != want)[0]
    pytest.fail(f"{name}: {len(bad)} of {len(which)} rows differ from the oracle; row {i}: "
                f"first differing subjects among the first {n}: "
                + str([(int(j), int(rows[k][j]), int(want[j])) for j in diff[:5]]))


def test_every_pair_plain_small():
    g, q, db, go, ge = golden("plain_small")
    d = swgb.Database.from_seqset(db)
    compare_rows("plain_small", g, d.search_plain(q.res, q.lens, go, ge), q, db, go, ge)
    plan = d.plan(len(q), q.total)
    compare_rows("plain_small", g, plan.search(q.res, q.lens, go, ge), q, db, go, ge)


def test_every_pair_paper_search():
    g, q, db, go, ge = golden("paper_search")
    d = swgb.Database.from_seqset(db)
    plan = d.plan(len(q), q.total)                       # the benchmark's plan
    compare_rows("paper_search", g, plan.search(q.res, q.lens, go, ge), q, db, go, ge)


def test_every_pair_batched_uneven_autotuned():
    from paper_2309_09609_gb300 import tune
    g, q, db, go, ge = golden("batched_uneven")
    d = swgb.Database.from_seqset(db)
    t = tune.tune(d, q, go, ge, cache=None, repeats=1)  # as the benchmark: autotuned, one graph
    plan = d.plan(len(q), q.total, **t["options"], use_graph=1)
    compare_rows("batched_uneven", g, plan.search(q.res, q.lens, go, ge), q, db, go, ge)


def test_every_pair_serving_trace():
    from paper_2309_09609_gb300 import serve
    g, q, db, go, ge = golden("serving_trace")
    d = swgb.Database.from_seqset(db)
    srv = serve.Server(d, gap_open=go, gap_extend=ge)    # the benchmark's server settings
    try:
        futs = [srv.submit(q.seq(i)) for i in range(len(q))]
        rows = [f.result(600) for f in futs]
    finally:
        srv.close()
    assert srv.report()["batches"] < len(q)              # requests were batched
    compare_rows("serving_trace", g, rows, q, db, go, ge)
