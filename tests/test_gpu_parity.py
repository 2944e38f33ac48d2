"""CUDA path vs the CPU oracle, bit-exact on every pair (integer scores).

Each case runs the library's paths through the C ABI -- the one-shot search,
a plan replaying its CUDA graph, and the plain int32 baseline -- and compares
every score with the oracle (Eq. 1-3).  Sizes span several tiles and ragged
tails: query lengths around the 16/32-row strips and the 256/512/1024-row intra
passes, subject lengths around the 8-residue chunks and the 64-subject groups.
"""
import numpy as np
import pytest

from helpers import concat, from_text, oracle_all, oracle_pairs, rand_matrix, seqset
from paper_2309_09609_gb300 import build as nvbuild
from paper_2309_09609_gb300 import swgb, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    nvbuild.build()
    swgb.lib()


def all_paths(q, db, go=10, ge=2, matrix=None, plain=True, **opts):
    """Scores through every path: the one-shot search, a plan (twice: the
    second replays its graph) with `opts`, the same plan forced to the
    one-query and to the two-query inter-task kernel and to the
    subject-pair and the two-query intra-task kernel, and the plain
    baseline.  Returns them with the stats of the `opts` plan."""
    d = swgb.Database.from_seqset(db)
    res = {"search": d.search(q.res, q.lens, go, ge, matrix)}
    p = d.plan(max(len(q), 1), max(q.total, 1), **opts)
    res["plan"] = p.search(q.res, q.lens, go, ge, matrix)
    st = p.stats()
    res["plan_replay"] = p.search(q.res, q.lens, go, ge, matrix)
    if "two_query" not in opts:
        for tq in (0, 2):
            pk = d.plan(max(len(q), 1), max(q.total, 1), two_query=tq, **opts)
            res[f"plan_two_query_{tq}"] = pk.search(q.res, q.lens, go, ge, matrix)
            if tq == 2 and len(q) >= 2 and st["inter_cells"] > 0 and not opts.get("force_int32"):
                assert pk.stats()["inter2_items"] > 0 and pk.stats()["inter_items"] == 0
    if "two_query_long" not in opts:
        for tq in (0, 2):
            pk = d.plan(max(len(q), 1), max(q.total, 1), two_query_long=tq, **opts)
            res[f"plan_two_query_long_{tq}"] = pk.search(q.res, q.lens, go, ge, matrix)
            if tq == 0:
                assert pk.stats()["pair2_items"] == 0
            elif len(q) >= 2 and st["inter_cells"] > 0 and st["intra_items"] > 0:
                assert pk.stats()["pair2_items"] > 0
    if plain:
        res["plain"] = d.search_plain(q.res, q.lens, go, ge, matrix)
    return res, st


def assert_exact(res, want):
    for name, got in res.items():
        assert got.shape == want.shape, name
        bad = np.argwhere(got != want)
        assert bad.size == 0, f"{name}: {len(bad)} pairs differ, first {bad[:5].tolist()} " \
                              f"got {got[tuple(bad[0])]} want {want[tuple(bad[0])]}"


def test_plain_small_workload():
    w = synth.plain_small(0)
    res, st = all_paths(w.queries, w.db)
    assert_exact(res, oracle_all(w.queries, w.db))
    assert st["cells"] == w.cells


@pytest.mark.parametrize("rows,cols", [(16, 4), (32, 4), (32, 8)])
@pytest.mark.parametrize("gaps", [(10, 2), (5, 1), (0, 1), (11, 1), (0, 0)])
def test_ragged_tiles(rows, cols, gaps):
    rng = np.random.default_rng(rows * 100 + gaps[0] * 7 + gaps[1])
    db = seqset(rng, list(range(0, 10)) + list(rng.integers(0, 300, size=503)))
    q = seqset(rng, [0, 1, 5, 15, 16, 17, 31, 32, 33, 250])
    res, _ = all_paths(q, db, *gaps, rows_per_thread=rows, inter_columns=cols)
    assert_exact(res, oracle_all(q, db, *gaps))


@pytest.mark.parametrize("rows", [16, 24, 32])
def test_two_query_streams_ragged(rows):
    # Thirteen queries around the strip height (and of length 0 and 1) dealt
    # to query streams: several stream pairs on a small database, queries
    # changing inside a half, empty halves padding the shorter stream.
    rng = np.random.default_rng(60 + rows)
    q = seqset(rng, [0, 1, 5, rows - 1, rows, rows + 1, 2 * rows, 3 * rows - 1, 100, 333, 47,
                     250, 8])
    db = concat(seqset(rng, [0, 1, 7, 8, 9, 63, 64, 65]), seqset(rng, rng.integers(1, 700, 300)))
    want = oracle_all(q, db)
    d = swgb.Database.from_seqset(db)
    res = {}
    for sub in (q, q.subset([3, 9, 10])):   # many stream pairs; one pair of two streams
        p = d.plan(len(sub), max(sub.total, 1), two_query=2, two_query_rows=rows)
        got = p.search(sub.res, sub.lens)
        st = p.stats()
        assert st["inter2_items"] > 0 and st["inter_items"] == 0
        res[len(sub)] = got
    assert_exact({"13": res[13]}, want)
    assert_exact({"3": res[3]}, want[[3, 9, 10]])


@pytest.mark.parametrize("rows", [16, 24, 32])
def test_two_query_saturation_in_one_half(rows):
    # a saturating query beside ordinary ones: its half is flagged and
    # recomputed, the other half of every word stays exact
    rng = np.random.default_rng(70 + rows)
    w = lambda k: "W" * k
    q = concat(from_text(w(2990), w(2978) + "A" * 40, "HEAGAWGHEE"), seqset(rng, [30, 500, 2000]))
    db = concat(from_text(w(2977), w(2978), w(3000) + "K" * 20), seqset(rng, rng.integers(1, 400, 200)))
    want = oracle_all(q, db)
    assert want.max() > 32767
    d = swgb.Database.from_seqset(db)
    p = d.plan(len(q), q.total, two_query=2, two_query_rows=rows, long_cutoff=4000)
    got = p.search(q.res, q.lens)
    assert p.stats()["recomputed_pairs"] >= 4 and p.stats()["inter2_items"] > 0
    assert_exact({"2q": got}, want)


@pytest.mark.parametrize("gaps", [(10, 2), (11, 1), (6, 3)])   # the two gap classes, general
def test_two_query_long_streams_ragged(gaps):
    # Long subjects scored two queries per word, one subject per warp:
    # thirteen queries around the 32-row strips and 1024-row passes (and of
    # length 0 and 1) in query streams, subjects around the 128-column residue
    # blocks; stream pairs chosen by the plan (here one query per stream) and
    # forced to one (queries changing inside a half, inside a pass).
    rng = np.random.default_rng(80 + gaps[1])
    q = seqset(rng, [0, 1, 31, 32, 33, 100, 1023, 1024, 1025, 2100, 57, 400, 7])
    lens = [101, 127, 128, 129, 255, 256, 257, 383, 384, 385, 1000, 2500]
    db = concat(seqset(rng, lens + list(rng.integers(150, 1200, 35))),
                seqset(rng, rng.integers(0, 100, 150)))
    want = oracle_all(q, db, *gaps)
    d = swgb.Database.from_seqset(db)
    for idx in (list(range(13)), [7, 9], [0, 1, 2], [9, 0, 5, 12, 6]):
        sub = q.subset(idx)
        groups = None                        # items of one stream pair: the subject groups
        for pairs in (1, 0):
            p = d.plan(len(sub), max(sub.total, 1), two_query_long=2, two_query_pairs=pairs,
                       long_cutoff=100)
            got = p.search(sub.res, sub.lens, *gaps)
            items = p.stats()["pair2_items"]
            groups = groups or items
            assert items > 0 and items % groups == 0
            assert_exact({f"{idx} pairs={pairs}": got}, want[idx])


def test_two_query_long_query_boundaries_at_pass_edges():
    # Forced to one stream pair, the streams are dealt longest first to the
    # shorter stream, so these batches put query boundaries at the edges of a
    # 1024-row pass: [2112, 1024, 1024] starts the third query at lane 0 of
    # the second pass in half 1 (half 0: one query of 66 strips, empty
    # strips after it); [1056, 992, 64] gives half 1 31 strips, then a query
    # of 2 strips across lane 31 of the first pass and lane 0 of the second;
    # [1000, 40 x 9] puts nine queries in half 1, several in one pass.
    rng = np.random.default_rng(90)
    db = concat(seqset(rng, list(rng.integers(130, 900, 20)) + [0, 0, 1, 128]),
                seqset(rng, rng.integers(1, 60, 20)))
    for lens in ([2112, 1024, 1024], [1056, 992, 64], [1000] + [40] * 9):
        q = seqset(rng, lens)
        want = oracle_all(q, db)
        d = swgb.Database.from_seqset(db)
        p = d.plan(len(q), q.total, two_query_long=2, two_query_pairs=1, long_cutoff=100)
        got = p.search(q.res, q.lens)
        assert p.stats()["pair2_items"] > 0
        assert_exact({str(lens): got}, want)


def test_two_query_long_small_group_and_empty_subjects():
    # every subject in one 64-subject group whose longest exceeds the
    # cutoff: the long part is all 13 subjects -- one item of 12 subjects and
    # one of a single subject (the other warps idle), two of length 0
    rng = np.random.default_rng(91)
    db = seqset(rng, [700, 300, 129, 0, 0, 5, 64, 1, 2, 900, 33, 17, 128])
    q = seqset(rng, [1, 40, 300, 1100, 77])
    d = swgb.Database.from_seqset(db)
    p = d.plan(len(q), q.total, two_query_long=2, long_cutoff=500)
    got = p.search(q.res, q.lens)
    assert p.stats()["pair2_items"] >= 2 and p.stats()["inter_cells"] == 0
    assert_exact({"small": got}, oracle_all(q, db))


def test_two_query_long_saturation_in_one_half():
    # saturating queries beside ordinary ones against long subjects: the
    # saturated half is flagged and recomputed, the other stays exact; one
    # stream pair, so a saturating query is followed by others in its half
    rng = np.random.default_rng(92)
    w = lambda k: "W" * k
    q = concat(from_text(w(2990), w(2978) + "A" * 40, "HEAGAWGHEE"), seqset(rng, [30, 500, 2000]))
    db = concat(from_text(w(2977), w(2978), w(3000) + "K" * 20),
                seqset(rng, rng.integers(200, 1500, 30)), seqset(rng, rng.integers(1, 90, 50)))
    want = oracle_all(q, db)
    assert want.max() > 32767
    d = swgb.Database.from_seqset(db)
    for pairs in (0, 1):
        p = d.plan(len(q), q.total, two_query_long=2, two_query_pairs=pairs, long_cutoff=100)
        got = p.search(q.res, q.lens)
        assert p.stats()["recomputed_pairs"] >= 4 and p.stats()["pair2_items"] > 0
        assert_exact({f"pairs={pairs}": got}, want)


def test_full_alphabet_and_asymmetric_matrix():
    rng = np.random.default_rng(3)
    m = rand_matrix(rng, -6, 9, symmetric=False)
    db = seqset(rng, rng.integers(1, 200, size=300), alpha=24)
    q = seqset(rng, [1, 7, 40, 77, 130], alpha=24)
    res, _ = all_paths(q, db, 6, 2, m)
    assert_exact(res, oracle_all(q, db, 6, 2, m.astype(np.int32)))


@pytest.mark.parametrize("intra_rows", [8, 16])
def test_long_subjects_intra_task(intra_rows):
    rng = np.random.default_rng(4 + intra_rows)
    # 150 long subjects (intra-task groups) and 130 of length <= 60 (inter-task groups)
    db = seqset(rng, list(rng.integers(1, 1500, size=150)) + [64, 65, 63, 1] +
                list(rng.integers(1, 61, size=130)))
    q = seqset(rng, [1, 31, 255, 256, 257, 300, 513, 700])
    res, st = all_paths(q, db, long_cutoff=64, intra_rows=intra_rows)
    assert st["intra_items"] > 0 and st["inter_items"] + st["inter2_items"] > 0
    # and every subject through the int32 intra-task kernel (several passes)
    d = swgb.Database.from_seqset(db)
    res["int32_intra"] = d.plan(len(q), q.total, force_int32=1, intra_rows=intra_rows).search(
        q.res, q.lens)
    assert_exact(res, oracle_all(q, db))


@pytest.mark.parametrize("gaps", [(10, 2), (11, 1), (6, 3)])   # the two gap classes, general
def test_packed_pairs_odd_count_and_unequal_lengths(gaps):
    # 65 long subjects: the last pair has one subject; pairs of unequal length
    rng = np.random.default_rng(40)
    db = seqset(rng, list(rng.integers(200, 2000, size=65)) + [7, 0, 150])
    q = seqset(rng, [1, 100, 511, 512, 513, 1100])
    res, st = all_paths(q, db, *gaps, long_cutoff=100, plain=False)
    assert st["intra_items"] >= 65 * len(q)
    assert_exact(res, oracle_all(q, db, *gaps))


def test_pair_kernel_widths_split_the_queries():
    # Long subjects are scored by pair_kernel<32> (1024-row passes) for the
    # queries whose padded cost is lower there -- here 513, 1000 and 3073
    # residues -- and by pair_kernel<16> (512-row passes) for the rest: 1,
    # 500, 1025, 1100 and 2049.  Both run several passes.
    rng = np.random.default_rng(42)
    db = seqset(rng, list(rng.integers(600, 2500, size=41)) + list(rng.integers(1, 300, size=70)))
    q = seqset(rng, [1, 500, 513, 1000, 1025, 1100, 2049, 3073])
    res, st = all_paths(q, db, long_cutoff=550, plain=False, two_query_long=0)
    assert st["intra_items"] >= 41 * len(q)
    assert_exact(res, oracle_all(q, db))


def test_pair_kernel_wide_subject_prefix():
    # More (pair, query) items than 16-row warps, so only the subject pairs
    # whose longer subject reaches wide_min_subject may go wide: the wide
    # kernel takes those pairs with the wide queries, the narrow one takes
    # them with the other queries, then every shorter pair with all queries.
    rng = np.random.default_rng(43)
    db = seqset(rng, list(rng.integers(600, 2000, size=700)) + list(rng.integers(1, 300, size=50)))
    q = seqset(rng, [513, 1000, 3073, 500, 1100, 700, 900, 2049])
    res, st = all_paths(q, db, long_cutoff=550, plain=False, wide_min_subject=1300,
                        two_query_long=0)
    assert st["intra_items"] >= 700 * len(q)
    assert_exact(res, oracle_all(q, db))


@pytest.mark.parametrize("wide_min_subject", [0, 1 << 30])
def test_overlapped_kernels(wide_min_subject):
    # overlap_kernels: the inter-task kernel runs alongside the two pair
    # kernels; same scores, and a saturated pair still goes to the recompute
    rng = np.random.default_rng(44)
    w = lambda k: "W" * k
    db = concat(from_text(w(2990), w(700)), seqset(rng, list(rng.integers(600, 2500, size=60)) +
                                                    list(rng.integers(1, 400, size=300))))
    q = concat(from_text(w(3000)), seqset(rng, [1, 300, 513, 1000, 2049, 3073]))
    want = oracle_all(q, db)
    res, st = all_paths(q, db, long_cutoff=550, plain=False, overlap_kernels=1,
                        wide_min_subject=wide_min_subject)
    assert st["recomputed_pairs"] >= 1 and st["intra_items"] > 0
    assert st["inter_items"] + st["inter2_items"] > 0
    assert_exact(res, want)


def test_saturation_through_the_pair_kernel():
    rng = np.random.default_rng(41)
    q = from_text("W" * 3100, "HEAGAWGHEE" * 30)
    db = concat(from_text("W" * 2990, "W" * 3050 + "A" * 30, "W" * 2000),
                seqset(rng, rng.integers(800, 3000, size=40)))
    want = oracle_all(q, db)
    assert want.max() > 32767
    res, st = all_paths(q, db, long_cutoff=500, plain=False)
    assert st["recomputed_pairs"] >= 2
    assert_exact(res, want)


def test_force_int32_everywhere():
    rng = np.random.default_rng(5)
    db = seqset(rng, rng.integers(0, 400, size=200))
    q = seqset(rng, [3, 100, 333])
    res, st = all_paths(q, db, force_int32=1)
    assert st["inter_items"] == 0
    assert_exact(res, oracle_all(q, db))


def test_saturation_is_recomputed_exactly():
    # runs of W score 11 each: 2977 -> 32747 stays in 16 bits, 2978 -> 32758
    # reaches the recompute threshold 32767 - 11, 3100 overflows
    rng = np.random.default_rng(6)
    w = lambda k: "W" * k
    q = from_text(w(3100), w(2978) + "A" * 50, "HEAGAWGHEE")
    subj = from_text(w(2977), w(2978), w(2990), w(3000) + "K" * 20, "PAWHEAE")
    filler = seqset(rng, rng.integers(10, 300, size=100))
    db = concat(subj, filler)
    want = oracle_all(q, db)
    assert want.max() > 32767
    res, st = all_paths(q, db, long_cutoff=4000)  # every group on the packed path
    assert st["recomputed_pairs"] >= 6
    assert_exact(res, want)


def test_saturation_with_eight_column_wavefront():
    # the 16-bit overflow guard and the int32 recompute with the inter-task
    # kernel's eight-column wavefront
    rng = np.random.default_rng(9)
    w = lambda k: "W" * k
    q = from_text(w(3100), w(2978) + "A" * 50, "HEAGAWGHEE")
    subj = from_text(w(2977), w(2978), w(2990), w(3000) + "K" * 20, "PAWHEAE")
    db = concat(subj, seqset(rng, rng.integers(10, 300, size=100)))
    want = oracle_all(q, db)
    res, st = all_paths(q, db, long_cutoff=4000, inter_columns=8)
    assert st["recomputed_pairs"] >= 6
    assert_exact(res, want)


def test_saturation_with_large_matrix_entries():
    rng = np.random.default_rng(7)
    m = rand_matrix(rng, -20, 10)
    np.fill_diagonal(m, 100)
    base = seqset(rng, [400])
    q = concat(base, seqset(rng, [50, 200]))
    db = concat(base, base, seqset(rng, rng.integers(5, 500, size=130)))
    want = oracle_all(q, db, 10, 2, m.astype(np.int32))
    assert want.max() > 32767
    res, st = all_paths(q, db, 10, 2, m)
    assert st["recomputed_pairs"] >= 2
    assert_exact(res, want)


def test_flag_list_overflow_is_recomputed_in_rounds():
    # Many saturated pairs against a flag list of 7 entries: the packed
    # kernels mark the pairs that find it full, and rounds of the int32
    # kernel after the search score them all exactly (through both the
    # inter-task and the pair kernels: the cutoff sends subjects over 300
    # residues to the latter).
    rng = np.random.default_rng(17)
    m = rand_matrix(rng, -20, 10)
    np.fill_diagonal(m, 120)
    base = seqset(rng, [420])
    homologs = [synth.mutate(rng, base.res, 0.03) for _ in range(90)]
    cut = [h[:int(k)] for h, k in zip(homologs, rng.integers(290, 421, 90))]
    db = concat(synth.SeqSet(np.concatenate(cut), np.array([c.size for c in cut], np.int32)),
                seqset(rng, rng.integers(5, 500, size=120)))
    q = concat(base, seqset(rng, [60]), synth.SeqSet(base.res[:380], np.array([380], np.int32)))
    want = oracle_all(q, db, 10, 2, m.astype(np.int32))
    # flagged exactly when S + Go reaches 32767 - max(SM) (Go = 12)
    n_sat = int((want + 12 >= 32767 - int(m.max())).sum())
    assert n_sat > 100
    d = swgb.Database.from_seqset(db)
    for opts in (dict(flag_capacity=7, long_cutoff=300), dict(flag_capacity=7, use_graph=0),
                 dict(flag_capacity=7, two_query=2), dict(flag_capacity=7, two_query=0),
                 dict(flag_capacity=7, long_cutoff=300, two_query_long=2)):
        p = d.plan(len(q), q.total, **opts)
        for _ in range(2):                                   # a plan reused after an overflow
            got = p.search(q.res, q.lens, 10, 2, m)          # scores to host memory
            st = p.stats()
            assert st["recomputed_pairs"] == n_sat and st["overflow_rounds"] >= 10
            assert_exact({"host": got}, want)
        torch = pytest.importorskip("torch")
        out = torch.full((len(q), len(db)), -5, dtype=torch.int32, device="cuda")
        p.search(q.res, q.lens, 10, 2, m, out=out)          # scores to device memory
        assert_exact({"device": out.cpu().numpy()}, want)


@pytest.mark.parametrize("intra_rows", [8, 16])
def test_recompute_spans_several_rounds_of_passes(intra_rows):
    # A flagged pair is recomputed by one block whose 16 warps take the query's
    # 32*TI-row passes in turn.  A 9,000-residue query has 36 (TI = 8) or 18
    # (TI = 16) passes, more than one round of warps.  The flagged subjects are
    # shorter (400: a pass lasts fewer stages than the 48 between a warp's
    # pass starts) and longer (2,000; 5,000) than that.
    rng = np.random.default_rng(70 + intra_rows)
    m = rand_matrix(rng, -20, 10)
    np.fill_diagonal(m, 100)
    q = seqset(rng, [9000, 700])
    q0 = q.seq(0)
    pieces = [q0[100:500], q0[3000:5000], q0[4000:9000], q0[8600:9000][::-1].copy()]
    flagged = synth.SeqSet(np.concatenate(pieces), np.array([p.size for p in pieces], np.int32))
    db = concat(flagged, seqset(rng, rng.integers(5, 600, size=70)))
    want = oracle_all(q, db, 10, 2, m.astype(np.int32))
    assert (want > 32767).sum() >= 3
    res, st = all_paths(q, db, 10, 2, m, intra_rows=intra_rows)
    assert st["recomputed_pairs"] >= 3
    assert_exact(res, want)


def test_huge_gap_penalties_take_the_int32_path():
    rng = np.random.default_rng(8)
    db = seqset(rng, rng.integers(0, 120, size=90))
    q = seqset(rng, [10, 64, 100])
    res, st = all_paths(q, db, 100000, 100000)
    assert st["inter_items"] == 0
    assert_exact(res, oracle_all(q, db, 100000, 100000))


def test_subject_permutation_permutes_columns():
    rng = np.random.default_rng(9)
    db = seqset(rng, rng.integers(0, 250, size=200))
    q = seqset(rng, [20, 90])
    perm = rng.permutation(len(db))
    db2 = db.subset(perm)
    d1, d2 = swgb.Database.from_seqset(db), swgb.Database.from_seqset(db2)
    a = d1.search(q.res, q.lens)
    b = d2.search(q.res, q.lens)
    assert (a[:, perm] == b).all()


def test_equal_lengths_and_cutoff_edges():
    rng = np.random.default_rng(10)
    db = concat(seqset(rng, [100] * 64), seqset(rng, [199, 200, 201, 8, 7, 9, 16]))
    q = seqset(rng, [17, 64])
    res, st = all_paths(q, db, long_cutoff=200)
    assert_exact(res, oracle_all(q, db))


def test_device_tensors_in_and_out():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    db = seqset(rng, rng.integers(1, 300, size=150))
    q = seqset(rng, [33, 120])
    d = swgb.Database.from_seqset(db)
    qt = torch.from_numpy(q.res).cuda()
    lt = torch.from_numpy(q.lens).cuda()
    out = torch.empty((len(q), len(db)), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    d.search(qt, lt, 10, 2, out=out, stream=stream)
    p = d.plan(4, 1000)
    out2 = torch.empty_like(out)
    p.search(qt, lt, 10, 2, out=out2, stream=stream)
    want = oracle_all(q, db)
    assert (out.cpu().numpy() == want).all()
    assert (out2.cpu().numpy() == want).all()


def test_plan_reuse_across_batches_and_scoring():
    rng = np.random.default_rng(12)
    db = seqset(rng, list(rng.integers(1, 600, size=300)) + [900, 1300])
    d = swgb.Database.from_seqset(db)
    p = d.plan(16, 8000, long_cutoff=800)
    m = rand_matrix(rng, -4, 6, symmetric=True)
    # gap settings of every class the packed kernels are compiled for --
    # (10, 2), (11, 1) and the general form -- alternate on one plan, which
    # keeps a CUDA graph per class
    batches = [
        (seqset(rng, [100, 7, 300]), 10, 2, None),
        (seqset(rng, [45] * 9 + [512]), 3, 1, m),
        (seqset(rng, [1]), 10, 2, None),
        (seqset(rng, [0, 0]), 10, 2, None),
        (seqset(rng, [250, 33, 700]), 11, 1, None),
        (seqset(rng, [250, 33, 700]), 10, 2, m),
        (seqset(rng, [250, 33, 700]), 9, 3, None),
        (seqset(rng, [250, 33, 700]), 11, 1, None),
    ]
    for q, go, ge, mm in batches:
        got = p.search(q.res, q.lens, go, ge, mm)
        want = oracle_all(q, db, go, ge, None if mm is None else mm.astype(np.int32))
        assert (got == want).all(), (go, ge)


def test_async_search_and_bounded_wait():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(13)
    db = seqset(rng, rng.integers(1, 500, size=4000))
    q = seqset(rng, [500, 800])
    d = swgb.Database.from_seqset(db)
    p = d.plan(2, 2000)
    out = torch.empty((2, len(db)), dtype=torch.int32, device="cuda")
    p.search_async(q.res, q.lens, out)
    p.wait(0)                      # a poll returns at once, finished or not
    assert p.wait(-1) is True
    assert p.wait(0) is True       # nothing in flight any more
    want = oracle_all(q, db)
    assert (out.cpu().numpy() == want).all()


def test_empty_inputs():
    rng = np.random.default_rng(14)
    db = seqset(rng, [0, 0, 5])
    d = swgb.Database.from_seqset(db)
    q = seqset(rng, [0, 4])
    assert (d.search(q.res, q.lens) == oracle_all(q, db)).all()
    assert d.search(np.zeros(0, np.uint8), np.zeros(0, np.int32)).shape == (0, 3)
    e = swgb.Database(np.zeros(0, np.uint8), np.zeros(0, np.int32))
    assert e.search(q.res, q.lens).shape == (2, 0)


def test_invalid_query_is_rejected_and_context_survives():
    rng = np.random.default_rng(15)
    db = seqset(rng, [10, 20])
    d = swgb.Database.from_seqset(db)
    with pytest.raises(swgb.SwError) as e:
        d.search(np.array([1, 2, 99], np.uint8), np.array([3], np.int32))
    assert e.value.status == swgb.SW_EINVAL
    with pytest.raises(swgb.SwError):
        d.search(np.array([1, 2], np.uint8), np.array([2], np.int32), -1, 2)
    p = d.plan(1, 4)
    with pytest.raises(swgb.SwError) as e:
        p.search(np.zeros(10, np.uint8), np.array([10], np.int32))
    assert e.value.status == swgb.SW_EBUSY
    q = seqset(rng, [5])
    assert (d.search(q.res, q.lens) == oracle_all(q, db)).all()
