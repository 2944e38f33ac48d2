"""The full-size workloads, in the launch configuration the benchmark times.

The oracle cannot score every pair at these sizes, so each test checks
(i) a random sample of pairs plus every planted homolog pair against the
oracle one by one, and (ii) properties that hold at any size: two independent
GPU paths (packed 16-bit inter-task vs plain int32, or vs the int32 intra-task
kernel) agree on every pair, and every score is >= 0.
"""
import numpy as np
import pytest

from helpers import oracle_pairs
from paper_2309_09609_gb300 import build as nvbuild
from paper_2309_09609_gb300 import swgb, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    nvbuild.build()
    swgb.lib()


def sample_pairs(rng, nq, nd, k, planted=()):
    pq = list(rng.integers(0, nq, k))
    pd = list(rng.integers(0, nd, k))
    for s in planted:
        for q in range(nq):
            pq.append(q)
            pd.append(int(s))
    return np.array(pq), np.array(pd)


def check_sample(got, w, pq, pd):
    want = oracle_pairs(w.queries, w.db, pq, pd, w.gap_open, w.gap_extend)
    bad = np.nonzero(got[pq, pd] != want)[0]
    assert bad.size == 0, [(int(pq[i]), int(pd[i]), int(got[pq[i], pd[i]]), int(want[i]))
                           for i in bad[:5]]
    return want


def test_paper_search_full_size():
    w = synth.paper_search(0)
    d = swgb.Database.from_seqset(w.db)
    plan = d.plan(len(w.queries), w.queries.total)           # the benchmark's plan
    got = plan.search(w.queries.res, w.queries.lens, w.gap_open, w.gap_extend)
    assert got.min() >= 0
    rng = np.random.default_rng(1)
    pq, pd = sample_pairs(rng, len(w.queries), len(w.db), 400, w.planted)
    want = check_sample(got, w, pq, pd)
    assert want.max() > 1000                                   # planted homologs score high
    plain = d.search_plain(w.queries.res, w.queries.lens, w.gap_open, w.gap_extend)
    assert (plain == got).all()


def test_batched_uneven_full_size_autotuned():
    from paper_2309_09609_gb300 import tune
    w = synth.batched_uneven(0)
    d = swgb.Database.from_seqset(w.db)
    t = tune.tune(d, w.queries, w.gap_open, w.gap_extend, cache=None, repeats=1)
    plan = d.plan(len(w.queries), w.queries.total, **t["options"], use_graph=1)
    got = plan.search(w.queries.res, w.queries.lens, w.gap_open, w.gap_extend)
    got2 = plan.search(w.queries.res, w.queries.lens, w.gap_open, w.gap_extend)  # graph replay
    assert (got == got2).all() and got.min() >= 0
    rng = np.random.default_rng(2)
    pq, pd = sample_pairs(rng, len(w.queries), len(w.db), 400, w.planted[:3])
    check_sample(got, w, pq, pd)
    # another tile shape gives the same scores
    other = d.plan(len(w.queries), w.queries.total, rows_per_thread=32, long_cutoff=1500)
    assert (other.search(w.queries.res, w.queries.lens, w.gap_open, w.gap_extend) == got).all()


def test_long_sequences_full_size():
    w = synth.long_sequences(0)
    d = swgb.Database.from_seqset(w.db)
    # the int32 intra-task warp-wavefront kernel for every subject
    intra = d.plan(len(w.queries), w.queries.total, force_int32=1, intra_rows=16)
    got = intra.search(w.queries.res, w.queries.lens, w.gap_open, w.gap_extend)
    st = intra.stats()
    assert st["inter_items"] == 0 and st["intra_items"] == len(w.queries) * len(w.db)
    assert got.max() > 32767                                   # int16 would saturate here
    rng = np.random.default_rng(3)
    pq, pd = sample_pairs(rng, len(w.queries), len(w.db), 6, w.planted)
    check_sample(got, w, pq, pd)
    # the packed intra-task kernel (subject pairs) with int32 recompute
    pairs = d.plan(len(w.queries), w.queries.total, long_cutoff=0)
    got2 = pairs.search(w.queries.res, w.queries.lens, w.gap_open, w.gap_extend)
    assert pairs.stats()["recomputed_pairs"] > 0 and pairs.stats()["inter_items"] == 0
    assert (got2 == got).all()
    # the packed inter-task kernel with int32 recompute
    packed = d.plan(len(w.queries), w.queries.total, long_cutoff=1 << 30, auto_cutoff=0)
    got3 = packed.search(w.queries.res, w.queries.lens, w.gap_open, w.gap_extend)
    assert packed.stats()["recomputed_pairs"] > 0
    assert (got3 == got).all()
