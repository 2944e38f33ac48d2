"""Host-side logic of bench.py that needs no GPU."""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _args(**kw):
    base = dict(workload="paper-search", subjects=None, queries=None, rows=None, warps=None,
                cutoff=None, tune=False, wide_min=None, wide_min_subject=None, two_query=None,
                two_query_rows=None)
    base.update(kw)
    return argparse.Namespace(**base)


def test_traffic_record_applies_only_to_the_profiled_kernel_and_workload():
    rec = bench.traffic_record()
    same = rec.get("kernel_sources_sha256") == bench.kernel_sources_sha256()
    t = bench.profiled_traffic(_args())
    if same:                                        # recorded for the current kernel sources
        assert isinstance(t, int) and t == int(rec["dram_bytes_per_launch"]) and t > 1e11
    else:                                           # kernel changed since the capture
        assert t is None
    assert bench.profiled_traffic(_args(subjects=1000)) is None
    assert bench.profiled_traffic(_args(rows=16)) is None
    assert bench.profiled_traffic(_args(cutoff=3000)) is None
    assert bench.profiled_traffic(_args(workload="long")) is None        # not the inter kernel's
    assert bench.profiled_traffic(_args(workload="batched-uneven"), "pair2q_kernel") is None
    assert bench.profiled_traffic(_args(), "inter_kernel") is None      # no record of that kernel
    assert bench.profiled_traffic(_args(workload="long"), "pair_kernel") is None
    assert bench.profiled_traffic(_args(two_query=0)) is None
    assert bench.profiled_traffic(_args(workload="long", two_query_long=0), "pair2q_kernel") is None
    long = bench.profiled_traffic(_args(workload="long"), "pair2q_kernel")
    path = os.path.join(ROOT, "profiles", bench.TRAFFIC_RECORDS[("pair2q_kernel", "long")][0])
    if os.path.exists(path):
        rec = bench.traffic_record(path)
        assert long is None or long == int(rec["dram_bytes_per_launch"])
    else:
        assert long is None


def test_workload_query_subset():
    w = bench.make_workload("plain-small", 0)
    assert len(w.queries) == 1 and len(w.db) == 2000
    w2 = bench.make_workload("paper-search", 0, subjects=2000, queries=3, query_offset=5)
    assert len(w2.db) == 2000 and len(w2.queries) == 3
    assert w2.queries.lens[0] == bench.make_workload("paper-search", 0, subjects=2000).queries.lens[5]


def test_oracle_sample_fits_the_cell_budget():
    for name in ("plain-small", "paper-search"):
        w = bench.make_workload(name, 0, subjects=5000 if name == "paper-search" else None)
        for budget in (1e6, 1e8, 1e9):
            sub = bench.oracle_sample(w, budget)
            cells = int(w.queries.total) * int(sub.total)
            assert len(sub) >= 1
            assert cells <= budget or len(sub) == 1
            if len(sub) < len(w.db):          # one more subject would not fit
                assert cells + int(w.queries.total) * int(w.db.lens[len(sub)]) > budget
            assert (sub.lens == w.db.lens[:len(sub)]).all()


def test_l2_note_follows_the_database_size():
    import bench
    assert "> 129 MB L2" in bench.l2_note(205_430_861)        # the paper-shaped database
    assert "fit in L2" in bench.l2_note(1_070_512)            # the small parity case


def test_paper_arch_efficiency_follows_eq5():
    import bench
    # Eq. 4-5 by hand: 46 SMs x 64 lane-ops per clock x 1725 MHz / 12 per cell
    r = bench.paper_arch_efficiency(280.2, 64.0, 46, 1725.0)
    assert abs(r["peak_gcups"] - 46 * 64 * 1725e6 / 12 / 1e9) < 0.1
    assert abs(r["value"] - 280.2 / (46 * 64 * 1725e6 / 12 / 1e9)) < 1e-4
    assert bench.paper_arch_efficiency(5965.0, 62.5, 152, 2070.0)["value"] > 1   # packed


def test_l2_flush_only_when_the_database_fits_in_l2():
    # two device layouts of about one byte per residue each
    assert bench.l2_flush_bytes(205_000_000) == 0                 # paper-shaped database
    assert bench.l2_flush_bytes(36_036_930) == 2 * bench.L2_BYTES  # batched-uneven database
    assert bench.l2_note(205_000_000).startswith("no flush")
    assert bench.l2_note(36_036_930).startswith("L2 flushed")


def test_roofline_names_the_dominant_kernel_and_counts_its_layouts_ops():
    # two-query layouts count 2.25 ALU lane-ops per cell, two-subject ones 2.75
    stats = {"inter2_items": 4, "pair2_items": 0, "cells": 10 ** 12, "inter_cells": 9 * 10 ** 11}
    t = {"stats": stats, "kernel_ms": [100.0, 100.0], "pair_ms": [20.0], "recompute_ms": [0.01]}
    r = bench.roofline(t, 20.0, "test", 2070.0, lambda k: 123 if k == "inter2q_kernel" else None)
    assert r["kernel"].startswith("inter2q_kernel") and r["traffic"] == 123
    assert r["alu_ops_per_cell"] == bench.TWO_QUERY_ALU_OPS_PER_CELL == 2.25
    assert abs(r["achieved"] - 2.25 * 9e11 / 0.1 / 1e12) < 1e-3 and abs(r["frac"] - r["achieved"] / 20.0) < 1e-4
    pair = r["kernels"]["pair_kernel (packed intra-task)"]
    assert pair["alu_ops_per_cell"] == bench.PACKED_ALU_OPS_PER_CELL == 2.75
    # the long workload: the pair kernel dominates, two queries per word
    stats = {"inter2_items": 0, "pair2_items": 8, "cells": 10 ** 12, "inter_cells": 0}
    t = {"stats": stats, "kernel_ms": [0.01], "pair_ms": [500.0], "recompute_ms": [5.0]}
    r = bench.roofline(t, 20.0, "test", 2070.0, lambda k: 7 if k == "pair2q_kernel" else None)
    assert r["kernel"].startswith("pair2q_kernel") and r["traffic"] == 7
    assert r["alu_ops_per_cell"] == 2.25 and r["pair_kernel_ms"] == 500.0
