"""Host-side logic of bench.py that needs no GPU."""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _args(**kw):
    base = dict(workload="paper-search", subjects=None, queries=None, rows=None, warps=None,
                cutoff=None, tune=False)
    base.update(kw)
    return argparse.Namespace(**base)


def test_traffic_record_applies_only_to_the_profiled_kernel_and_workload():
    t = bench.profiled_traffic(_args())
    assert isinstance(t, int) and t > 1e11          # recorded for the current kernel source
    assert bench.profiled_traffic(_args(subjects=1000)) is None
    assert bench.profiled_traffic(_args(rows=16)) is None
    assert bench.profiled_traffic(_args(cutoff=3000)) is None
    assert bench.profiled_traffic(_args(workload="long")) is None


def test_workload_query_subset():
    w = bench.make_workload("plain-small", 0)
    assert len(w.queries) == 1 and len(w.db) == 2000
    w2 = bench.make_workload("paper-search", 0, subjects=2000, queries=3, query_offset=5)
    assert len(w2.db) == 2000 and len(w2.queries) == 3
    assert w2.queries.lens[0] == bench.make_workload("paper-search", 0, subjects=2000).queries.lens[5]
