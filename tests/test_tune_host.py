"""The autotuner's candidate set, on the CPU: every option set is one the plan
accepts, none is listed twice, and settings that cannot differ collapse."""
import json
import types

from paper_2309_09609_gb300 import tune


def _db(max_length):
    return types.SimpleNamespace(max_length=max_length)


def _valid(o):
    return (o["rows_per_thread"] in (16, 32) and o["warps_per_block"] in (4, 8)
            and o["intra_rows"] in (8, 16) and o["inter_columns"] in (4, 8)
            and (o["rows_per_thread"] == 32 or o["inter_columns"] == 4))


def test_candidates_for_a_database_with_long_subjects():
    c = tune.candidates(_db(35000))
    assert all(_valid(o) for o in c)
    keys = {tuple(sorted(o.items())) for o in c}
    # (three real cutoffs x two int32 row counts + "no cutoff" with one)
    # x (rows 16 with 4 columns + rows 32 with 4 or 8) x two warp counts
    assert len(keys) == len(c) == 7 * 3 * 2
    assert sorted({o["long_cutoff"] for o in c}) == [1500, 3000, 7000, 1 << 30]
    assert {o["intra_rows"] for o in c if o["long_cutoff"] == 1 << 30} == {8}


def test_cutoffs_at_or_above_the_longest_subject_collapse():
    # a longest subject between 3000 and 7000 (the batched workload's case)
    mid = tune.candidates(_db(5000))
    assert sorted({o["long_cutoff"] for o in mid}) == [1500, 3000, 1 << 30]
    assert len(mid) == 5 * 3 * 2 == 30
    c = tune.candidates(_db(2000))
    assert sorted({o["long_cutoff"] for o in c}) == [1500, 1 << 30]
    short = tune.candidates(_db(1000))
    assert {o["long_cutoff"] for o in short} == {1 << 30}
    # rows 16 (4 columns) and rows 32 (4 or 8 columns), two warp counts each
    assert len(short) == 2 * (1 + 2)
    assert all(_valid(o) for o in short)


def test_cache_file_that_is_missing_or_corrupt_reads_as_empty(tmp_path):
    assert tune._load(str(tmp_path / "absent.json")) == {}
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    assert tune._load(str(bad)) == {}
    good = tmp_path / "good.json"
    good.write_text(json.dumps({"k": {"options": {"rows_per_thread": 32}}}))
    assert tune._load(str(good))["k"]["options"]["rows_per_thread"] == 32
