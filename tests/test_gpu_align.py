"""sw_align (optimal local alignment with traceback) vs the CPU oracle:
score, end points and transcript identical pair by pair.  The oracle and the
library follow the same stated rules for which optimal alignment to return,
so the whole alignment is compared, not only its score."""
import ctypes

import numpy as np
import pytest

from helpers import concat, from_text, oracle_all, rand_matrix, seqset
import oracle
from paper_2309_09609_gb300 import build as nvbuild
from paper_2309_09609_gb300 import swgb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    nvbuild.build()
    swgb.lib()


def check(q, db, pq, ps, gaps=(10, 2), matrix=None):
    d = swgb.Database.from_seqset(db)
    got = d.align(q.res, q.lens, pq, ps, *gaps, matrix)
    sm = None if matrix is None else np.asarray(matrix, dtype=np.int32)
    for k, (a, b) in enumerate(zip(pq, ps)):
        want = oracle.align(q.seq(int(a)), db.seq(int(b)), *gaps, sm)
        assert got[k] == want, f"pair {k} (query {a}, subject {b}): {got[k]} != {want}"
    return got


def test_random_pairs_with_planted_homologs():
    rng = np.random.default_rng(11)
    q = seqset(rng, [1, 37, 255, 256, 257, 600, 1100])
    db = seqset(rng, rng.integers(0, 700, size=60))
    # plant a mutated copy of part of each query into a subject
    res, lens = db.res.copy(), db.lens
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]])
    for a in range(len(q)):
        src = q.seq(a)
        k = 3 * a + 1
        L = min(len(src), int(lens[k]))
        if L > 10:
            seg = src[:L].copy()
            seg[::7] = (seg[::7] + 3) % 20
            res[offs[k]:offs[k] + L] = seg
    db.res = res
    pq = np.repeat(np.arange(len(q)), 8)
    ps = np.concatenate([rng.choice(len(db), 7, replace=False).tolist() + [3 * a + 1]
                         for a in range(len(q))])
    got = check(q, db, pq, ps)
    assert any(len(g["ops"]) > 50 for g in got)


@pytest.mark.parametrize("alpha", [2, 3])
def test_many_ties_small_alphabet(alpha):
    rng = np.random.default_rng(20 + alpha)
    m = rand_matrix(rng, -3, 3)
    q = seqset(rng, rng.integers(1, 90, size=12), alpha=alpha)
    db = seqset(rng, rng.integers(1, 90, size=40), alpha=alpha)
    pq = np.repeat(np.arange(len(q)), 5)
    ps = rng.integers(0, len(db), size=pq.size)
    for gaps in [(2, 1), (0, 1), (0, 0), (3, 3)]:
        check(q, db, pq, ps, gaps, m)


def test_many_pairs_one_warp_each():
    # more pairs than SMs: one warp per pair (fewer pairs get a block each,
    # as in the other tests); both must give the same alignments
    rng = np.random.default_rng(16)
    q = seqset(rng, rng.integers(1, 400, size=20))
    db = seqset(rng, rng.integers(1, 400, size=40))
    pq = np.repeat(np.arange(len(q)), 20)
    ps = rng.integers(0, len(db), size=pq.size)
    got = check(q, db, pq, ps)
    assert len(got) == 400
    d = swgb.Database.from_seqset(db)
    assert d.align(q.res, q.lens, pq[:5], ps[:5]) == got[:5]       # block per pair


def test_scores_equal_the_search_and_zero_scores():
    rng = np.random.default_rng(12)
    q = concat(seqset(rng, [0, 5, 300]), from_text("PPPP"))
    db = concat(seqset(rng, rng.integers(0, 400, size=30)), from_text("", "WWWW"))
    m = np.full((24, 24), -1, np.int8)   # nothing scores > 0: every score is 0
    pq = np.repeat(np.arange(len(q)), len(db))
    ps = np.tile(np.arange(len(db)), len(q))
    got = check(q, db, pq, ps)
    d = swgb.Database.from_seqset(db)
    scores = d.search(q.res, q.lens, 10, 2)
    assert [g["score"] for g in got] == scores.reshape(-1).tolist()
    zero = check(q, db, pq, ps, (10, 2), m)
    assert all(g == {"score": 0, "q_begin": 0, "q_end": 0, "s_begin": 0, "s_end": 0, "ops": ""}
               for g in zero)


def test_long_pair_several_passes():
    rng = np.random.default_rng(13)
    base = seqset(rng, [3000]).seq(0)
    mut = base.copy()
    mut[::11] = (mut[::11] + 5) % 20
    q = concat(from_text("HEAGAWGHEE"), seqset(rng, [1800]))
    q.res = np.concatenate([q.res[:10], base[:1800]])
    db = seqset(rng, [2500, 40])
    db.res = np.concatenate([np.delete(mut[:2520], np.arange(300, 320)), db.res[2500:]])
    got = check(q, db, [1, 1, 0], [0, 1, 0])
    assert got[0]["ops"].count("I") >= 20    # the deleted stretch is a query-side gap


def test_bad_arguments_are_rejected():
    rng = np.random.default_rng(14)
    q = seqset(rng, [10, 20])
    db = seqset(rng, [30, 40])
    d = swgb.Database.from_seqset(db)
    with pytest.raises(swgb.SwError) as e:
        d.align(q.res, q.lens, [0, 2], [0, 1])
    assert e.value.status == swgb.SW_EINVAL
    L = swgb.lib()
    out = (swgb.Alignment * 1)()
    ops = np.zeros(10, np.uint8)
    pq, ps = np.array([0], np.int32), np.array([5], np.int64)
    st = L.sw_align(d._h, swgb._ptr(q.res), swgb._ptr(q.lens), 2, swgb._ptr(pq), swgb._ptr(ps), 1,
                    10, 2, None, out, swgb._ptr(ops), ops.size, None)
    assert st == swgb.SW_EINVAL and "subject" in swgb.last_error()
    ps = np.array([1], np.int64)
    st = L.sw_align(d._h, swgb._ptr(q.res), swgb._ptr(q.lens), 2, swgb._ptr(pq), swgb._ptr(ps), 1,
                    10, 2, None, out, swgb._ptr(ops), ops.size, None)   # needs 10 + 40 bytes
    assert st == swgb.SW_EINVAL and "ops needs" in swgb.last_error()
    assert d.align(q.res, q.lens, [], []) == []
    # the context is still usable
    assert d.align(q.res, q.lens, [1], [1])[0]["score"] == oracle_all(q, db)[1, 1]


def test_full_size_pair_by_properties():
    # A 20,000 x 25,000 pair (79 passes, 0.25 GB of direction bits): too big
    # for the full-matrix oracle, so the alignment is checked by properties
    # that fix it at any size, with the linear-space score oracle.
    from test_oracle_align_pins import rescore
    rng = np.random.default_rng(15)
    q = seqset(rng, [20000])
    core = q.seq(0)[2000:17000].copy()
    core[::9] = (core[::9] + 7) % 20                        # substitutions
    core = np.delete(core, np.arange(5000, 5012))          # a 12-residue deletion
    core = np.insert(core, 9000, rng.integers(0, 20, 30).astype(np.uint8))  # an insertion
    d_seq = np.concatenate([rng.integers(0, 20, 4000), core, rng.integers(0, 20, 6018)])
    db = seqset(rng, [len(d_seq)])
    db.res = d_seq.astype(np.uint8)
    d = swgb.Database.from_seqset(db)
    a = d.align(q.res, q.lens, [0], [0])[0]
    qs, ds = q.seq(0), db.seq(0)
    s = oracle.sw_score(qs, ds)
    assert a["score"] == s and s > 20000
    assert rescore(qs, ds, a, oracle.blosum62(), 10, 2) == s
    assert oracle.sw_score(qs[a["q_begin"]:a["q_end"]], ds[a["s_begin"]:a["s_end"]]) == s
    assert oracle.sw_score(qs[:a["q_end"] - 1], ds) < s
    assert oracle.sw_score(qs[:a["q_end"]], ds[:a["s_end"] - 1]) < s
    assert a["ops"].count("I") >= 10 and a["ops"].count("D") >= 10   # both indels are gaps
