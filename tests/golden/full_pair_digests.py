"""Writes every-pair score digests of the full-size workloads, from the oracle only.

For each query row of a workload's score matrix (every subject, caller order)
the oracle (Eq. 1-3, BLOSUM62, gap cost 10 + 2k) computes all scores on the
host cores, and this script stores the row's SHA-256 (int32 little-endian),
its maximum and its sum.  A GPU test recomputes the same digests from the
library's scores, so that every pair of these workloads is compared, not a
sample.  The workload inputs are redrawn from their seeds by ``synth``; the
header keeps a SHA-256 of those inputs so that a different draw is reported
as such.

Usage (takes CPU hours for the larger workloads; resumable)::

    python tests/golden/full_pair_digests.py plain_small paper_search serving_trace ...

Output: ``tests/golden/full_pairs_<name>.txt``.  Rows already computed are kept
in ``full_pairs_<name>.txt.partial`` until the file is complete, and a rerun
continues from there.
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2309_09609_gb300 import synth  # noqa: E402  (input generators only)

#: arrivals of the serving trace whose rows are stored (a prefix of the
#: 1,000-arrival trace the benchmark replays)
SERVING_ROWS = 100
SERVING_TRACE_LEN = 1000


def workload(name: str):
    """(queries, database, gap_open, gap_extend, description) of a named workload."""
    if name == "plain_small":
        w = synth.plain_small(0)
    elif name == "paper_search":
        w = synth.paper_search(0)
    elif name == "batched_uneven":
        w = synth.batched_uneven(0)
    elif name == "long_sequences":
        w = synth.long_sequences(0)
    elif name == "serving_trace":
        db = synth.paper_search(0).db
        tr = synth.serving_trace(0, n=SERVING_TRACE_LEN)
        q = tr.queries.subset(np.arange(SERVING_ROWS))
        return (q, db, 10, 2, f"serving trace (seed 0, {SERVING_TRACE_LEN} arrivals at 50/s), "
                f"arrivals 0..{SERVING_ROWS - 1} vs the paper-search database (seed 0)")
    else:
        raise ValueError(f"unknown workload {name!r}")
    return w.queries, w.db, w.gap_open, w.gap_extend, f"{w.name} (seed 0)"


def input_digest(q, db, gap_open: int, gap_extend: int) -> str:
    """SHA-256 of the inputs: query and subject lengths and codes, and the gaps."""
    h = hashlib.sha256()
    for a in (q.lens, q.res, db.lens, db.res):
        h.update(np.ascontiguousarray(a).tobytes())
    h.update(np.array([gap_open, gap_extend], dtype="<i4").tobytes())
    return h.hexdigest()


def row_digest(row) -> tuple[int, int, str]:
    """(max, sum, SHA-256 of the int32 little-endian bytes) of one score row."""
    r = np.ascontiguousarray(np.asarray(row), dtype="<i4")
    return (int(r.max()) if r.size else 0, int(r.sum(dtype=np.int64)),
            hashlib.sha256(r.tobytes()).hexdigest())


def read(path: str) -> dict:
    """Parses a digest file: header fields and {query index: (length, max, sum, sha)}."""
    head, rows = {}, {}
    with open(path) as f:
        for line in f:
            line = line.rstrip("\n")
            if line.startswith("#"):
                if ":" in line:
                    k, v = line[1:].split(":", 1)
                    head[k.strip()] = v.strip()
                continue
            if not line.strip():
                continue
            i, m, mx, sm, sha = line.split()
            rows[int(i)] = (int(m), int(mx), int(sm), sha)
    return {"head": head, "rows": rows}


def path_of(name: str) -> str:
    return os.path.join(HERE, f"full_pairs_{name}.txt")


def write(name: str, threads: int) -> None:
    import oracle  # the only scorer this script calls
    q, db, go, ge, desc = workload(name)
    digest = input_digest(q, db, go, ge)
    out = path_of(name)
    part = out + ".partial"
    done = {}
    if os.path.exists(part):
        prev = read(part)
        if prev["head"].get("input_sha256") == digest:
            done = prev["rows"]
    header = [
        "# Every-pair Smith-Waterman/Gotoh scores (Section II-B, Eq. 1-3), one digest per query row",
        "# written by tests/golden/full_pair_digests.py, which calls only the oracle",
        f"# workload: {desc}",
        f"# queries: {len(q)}",
        f"# subjects: {len(db)}",
        f"# cells: {q.total * db.total}",
        f"# gap_open: {go}",
        f"# gap_extend: {ge}",
        "# matrix: BLOSUM62",
        f"# input_sha256: {digest}",
        "# columns: query_index query_length row_max row_sum row_sha256 (int32 little-endian, caller order)",
    ]
    with open(part, "w") as f:
        f.write("\n".join(header) + "\n")
        for i in sorted(done):
            m, mx, sm, sha = done[i]
            f.write(f"{i} {m} {mx} {sm} {sha}\n")
    nd = len(db)
    pd = np.arange(nd, dtype=np.int64)
    t0 = time.time()
    cells = 0
    for i in range(len(q)):
        if i in done:
            continue
        pq = np.full(nd, i, dtype=np.int32)
        row = oracle.pairs_packed(q.res, q.offs, q.lens, db.res, db.offs, db.lens, pq, pd,
                                  go, ge, None, threads)
        mx, sm, sha = row_digest(row)
        with open(part, "a") as f:
            f.write(f"{i} {int(q.lens[i])} {mx} {sm} {sha}\n")
        cells += int(q.lens[i]) * db.total
        el = time.time() - t0
        print(f"{name}: row {i + 1}/{len(q)}  {cells / max(el, 1e-9) / 1e9:.2f} GCUPS  {el:.0f} s",
              flush=True)
    os.replace(part, out)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("names", nargs="+")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    for n in a.names:
        write(n, a.threads)


if __name__ == "__main__":
    main()
