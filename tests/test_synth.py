"""The seeded input generators: shapes, distributions and planted homologs."""
import numpy as np

from paper_2309_09609_gb300 import synth


def test_background_frequencies():
    f = synth.BACKGROUND
    assert f.size == 20 and abs(f.sum() - 1.0) < 1e-9
    x = synth.residues(np.random.default_rng(0), 2_000_000)
    assert x.max() < 20
    emp = np.bincount(x, minlength=20) / x.size
    assert np.abs(emp - f).max() < 1e-3


def test_lognormal_lengths_match_the_database_shape():
    L = synth.lognormal_lengths(np.random.default_rng(1), 400_000)
    assert L.min() >= 2 and L.max() <= 35000
    assert abs(L.mean() - 360) < 3 and abs(np.median(L) - 290) < 3


def test_paper_query_lengths():
    q = synth.paper_query_lengths()
    assert q[0] == 144 and q[-1] == 5478 and q.size == 20
    assert (np.diff(q) > 0).all()


def test_plant_homologs_keeps_lengths_and_copies_segments():
    rng = np.random.default_rng(2)
    src = synth.random_seqset(rng, [500, 800])
    db = synth.random_seqset(rng, [100, 900, 300, 50])
    lens = db.lens.copy()
    idx = synth.plant_homologs(rng, db, src, 4, 0.0, 0.0)
    assert (db.lens == lens).all() and sorted(idx) == [0, 1, 2, 3]
    whole = [src.seq(0).tobytes(), src.seq(1).tobytes()]
    for i in range(4):
        s = db.seq(i).tobytes()
        # a window of a source (short subject) or a source embedded in it (long subject)
        assert any(s in w or w in s for w in whole)


def test_workload_shapes_are_seeded():
    a = synth.plain_small(0)
    b = synth.plain_small(0)
    assert (a.db.res == b.db.res).all() and len(a.db) == 2000 and a.queries.total == 144
    assert 50 <= a.db.lens.min() and a.db.lens.max() <= 1000
    t = synth.serving_trace(0, n=500)
    assert (np.diff(t.times) >= 0).all() and 30 <= t.queries.lens.min()
    assert t.queries.lens.max() <= 5000
    assert 6.0 < t.times[-1] < 14.0          # 500 arrivals at 50 per second
    assert abs(t.queries.lens.mean() - 400) < 40


def test_tuner_sample_spans_query_lengths():
    from paper_2309_09609_gb300 import tune
    rng = np.random.default_rng(3)
    q = synth.random_seqset(rng, rng.integers(50, 2000, size=200))
    s, idx = tune.sample_queries(q, 8)
    assert len(s) == 8
    assert s.lens.min() == q.lens.min() and s.lens.max() == q.lens.max()
