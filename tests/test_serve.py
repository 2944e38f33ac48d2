"""Serving loop: continuous batching over stream slots, memory-bounded
admission, and identical results alone and in a mix."""
import numpy as np
import pytest

from helpers import oracle_all, oracle_pairs, seqset
from paper_2309_09609_gb300 import build as nvbuild
from paper_2309_09609_gb300 import swgb, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def db():
    nvbuild.build()
    rng = np.random.default_rng(21)
    ss = synth.random_seqset(rng, synth.lognormal_lengths(rng, 20000))
    return ss, swgb.Database.from_seqset(ss)


def test_results_alone_equal_results_in_the_mix(db):
    from paper_2309_09609_gb300 import serve
    ss, d = db
    trace = synth.serving_trace(seed=3, n=60, rate=2000.0)
    srv = serve.Server(d, slots=3, max_batch=8, max_batch_residues=20000)
    try:
        futs = serve.replay(srv, trace)
    finally:
        srv.close()
    rep = srv.report()
    assert rep["requests"] == 60 and rep["batches"] < 60      # requests were batched
    assert rep["max_concurrent_batches"] >= 2                 # batches overlapped
    mixed = [f.result() for f in futs]
    for i in range(len(trace.queries)):
        q = trace.queries.seq(i)
        alone = d.search(q, np.array([q.size], np.int32))[0]
        assert (mixed[i] == alone).all(), i
    # and a sample of pairs against the oracle
    rng = np.random.default_rng(0)
    qi = rng.integers(0, len(trace.queries), 40)
    di = rng.integers(0, len(ss), 40)
    want = oracle_pairs(trace.queries, ss, qi, di)
    got = np.array([mixed[a][b] for a, b in zip(qi, di)])
    assert (got == want).all()


def test_admission_refuses_what_can_never_fit(db):
    from paper_2309_09609_gb300 import serve
    ss, d = db
    srv = serve.Server(d, slots=1, max_batch=2, max_batch_residues=1000,
                       memory_budget=d.n * 13)
    try:
        with pytest.raises(serve.AdmissionError):
            srv.submit(np.zeros(2000, np.uint8))          # more residues than a batch holds
        with pytest.raises(ValueError):
            srv.submit(np.array([1, 2, 40], np.uint8))     # bad residue code
        q = seqset(np.random.default_rng(1), [100]).res
        assert srv.submit(q).result(60).shape == (d.n,)    # the server still works
    finally:
        srv.close()
    small = serve.Server(d, slots=1, max_batch=2, max_batch_residues=1000, memory_budget=100)
    try:
        with pytest.raises(serve.AdmissionError):
            small.submit(np.zeros(10, np.uint8))           # budget below one scores row
    finally:
        small.close()


def test_a_budget_below_the_offered_load_holds_requests_back(db):
    """Twelve requests offered at once against a budget of two: at most two
    are admitted at any time, the rest wait, and every score row equals the
    oracle's on every subject."""
    from paper_2309_09609_gb300 import serve
    ss, d = db
    rng = np.random.default_rng(4)
    qs = seqset(rng, rng.integers(40, 151, 12))
    srv = serve.Server(d, slots=2, max_batch=8, max_batch_residues=20000)
    budget = 2 * srv.request_bytes(int(qs.lens.max()))
    srv.close()
    srv = serve.Server(d, slots=2, max_batch=8, max_batch_residues=20000, memory_budget=budget)
    assert srv.free_at_start is not None and srv.free_at_start > budget
    try:
        with srv._lock:     # all twelve queued before the scheduler looks
            futs = [srv.submit(qs.seq(i)) for i in range(len(qs))]
        rows = np.stack([f.result(120) for f in futs])
    finally:
        srv.close()
    assert srv.max_in_use <= budget
    assert srv.report()["batches"] >= 6                 # never more than two per batch
    assert max(sum(1 for r in srv.completed if r.batch == b)
               for b in {r.batch for r in srv.completed}) <= 2
    assert (rows == oracle_all(qs, ss)).all()
