"""The autotuner's search, on the CPU: the option space, the constraint
between options, and the coordinate descent against cost functions whose
optimum is known."""
import itertools
import json
import types

import pytest

from paper_2309_09609_gb300 import tune


def _db(max_length):
    return types.SimpleNamespace(max_length=max_length)


def test_space_collapses_what_cannot_differ():
    sp = tune.space(_db(35000), 20)
    assert list(sp)[0] == "two_query" and "two_query_rows" not in sp
    assert sp["long_cutoff"] == [1500, 3000, 7000, tune.NO_CUTOFF]
    assert sp["intra_rows"] == [8, 16]
    assert all(len(set(v)) == len(v) for v in sp.values())
    mid = tune.space(_db(5000), 1000)
    assert mid["long_cutoff"] == [1500, 3000, tune.NO_CUTOFF]
    short = tune.space(_db(1000), 1)          # one query, no long subjects
    assert short["long_cutoff"] == [tune.NO_CUTOFF]
    assert "intra_rows" not in short and "two_query" not in short
    # the defaults come first and are those of the library
    assert {k: v[0] for k, v in sp.items()} == {
        "two_query": 1, "rows_per_thread": 32, "inter_columns": 8,
        "warps_per_block": 8, "long_cutoff": 1500, "intra_rows": 8}


def test_valid_needs_32_rows_for_eight_columns():
    assert tune.valid({"rows_per_thread": 32, "inter_columns": 8})
    assert tune.valid({"rows_per_thread": 16, "inter_columns": 4})
    assert not tune.valid({"rows_per_thread": 16, "inter_columns": 8})


@pytest.mark.parametrize("target", [
    {"two_query": 0, "rows_per_thread": 16, "inter_columns": 4,
     "warps_per_block": 4, "long_cutoff": 3000, "intra_rows": 16},
    {"two_query": 1, "rows_per_thread": 32, "inter_columns": 8,
     "warps_per_block": 8, "long_cutoff": tune.NO_CUTOFF, "intra_rows": 8},
])
def test_descent_finds_the_optimum_of_a_separable_cost(target):
    sp = tune.space(_db(35000), 20)
    calls = []

    def measure(opt):
        calls.append(dict(opt))
        assert tune.valid(opt)
        return sum(1.0 + (opt[k] != target[k]) * (1 + i) for i, k in enumerate(sorted(opt)))

    best, timings = tune.descend(sp, measure)
    assert best == target
    keys = [tuple(sorted(c.items())) for c in calls]
    assert len(keys) == len(set(keys))                 # nothing timed twice
    full = sum(1 for combo in itertools.product(*sp.values())
               if tune.valid(dict(zip(sp, combo))))
    assert len(calls) < full / 4                       # far fewer than the full product
    assert [t[0] for t in timings] == calls


def test_descent_skips_shapes_that_cannot_run_and_keeps_the_default_when_best():
    sp = tune.space(_db(5000), 4)
    best, timings = tune.descend(sp, lambda o: None if o["warps_per_block"] == 4 else 1.0)
    assert best == {k: v[0] for k, v in sp.items()}
    assert all(o["warps_per_block"] == 8 for o, _ in timings)
    with pytest.raises(RuntimeError):
        tune.descend(sp, lambda o: None)


def test_cache_file_that_is_missing_or_corrupt_reads_as_empty(tmp_path):
    assert tune._load(str(tmp_path / "absent.json")) == {}
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    assert tune._load(str(bad)) == {}
    good = tmp_path / "good.json"
    good.write_text(json.dumps({"k": {"options": {"rows_per_thread": 32}}}))
    assert tune._load(str(good))["k"]["options"]["rows_per_thread"] == 32
