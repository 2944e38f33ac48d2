"""Autotuner for the search plan's tile shape.

Candidates: query rows per thread of the packed kernel (16, 32), columns per
wavefront with 32 rows (4, 8), warps per block (4, 8), the inter/intra length
cutoff, and rows per lane of the int32 intra-task kernel (8, 16).  None of
them changes a score; they change speed only.  Each candidate runs a plan
over a length-stratified sample of the batch's queries against the whole
resident database and is timed by the plan's own CUDA events around all of
its kernels (pair, inter-task and recompute).  The best is cached in a JSON
file keyed by GPU, SM count, database signature, the sample's query length
profile and the gap penalties.
"""
from __future__ import annotations

import itertools
import json
import os
import threading

import numpy as np

from . import swgb

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "swgb", "tune.json")
ROWS = (16, 32)
WARPS = (4, 8)
CUTOFFS = (1500, 3000, 7000, 1 << 30)
INTRA_ROWS = (8, 16)
COLS = (4, 8)
_lock = threading.Lock()


def sample_queries(queries, k: int = 8):
    """Up to k queries at evenly spaced length quantiles of the batch."""
    n = len(queries)
    if n <= k:
        return queries, np.arange(n)
    order = np.argsort(queries.lens, kind="stable")
    idx = order[np.unique(np.linspace(0, n - 1, k).round().astype(int))]
    return queries.subset(idx), idx


def candidates(db: swgb.Database, rows=ROWS, warps=WARPS, cutoffs=CUTOFFS, intra_rows=INTRA_ROWS,
               cols=COLS):
    """Distinct option sets: cutoffs at or above the longest subject are one,
    and 16 rows per thread have one column count (4)."""
    maxlen = db.max_length
    cuts = sorted({c if c < maxlen else 1 << 30 for c in cutoffs})
    out = []
    for r, w, c in itertools.product(rows, warps, cuts):
        irs = intra_rows if c < maxlen else intra_rows[:1]
        for ir in irs:
            for k in (cols if r == 32 else (4,)):
                out.append(dict(rows_per_thread=r, warps_per_block=w, long_cutoff=c, intra_rows=ir,
                                inter_columns=k))
    return out


def _key(db, sample, gap_open, gap_extend) -> str:
    import torch
    dev = torch.cuda.get_device_properties(db.device)
    ql = np.sort(sample.lens)
    bucket = ",".join(str(int(2 ** round(np.log2(max(x, 1))))) for x in ql)
    return (f"{dev.name}|sm{dev.multi_processor_count}|db{db.n}:{db.residues}:{db.max_length}|"
            f"q[{bucket}]|g{gap_open},{gap_extend}")


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def tune(db: swgb.Database, queries, gap_open: int = 10, gap_extend: int = 2,
         cands=None, repeats: int = 2, cache: str | None = DEFAULT_CACHE, sample_size: int = 8):
    """Returns {"options": best option dict, "timings": [(options, ms), ...],
    "key": cache key, "cached": bool}."""
    import torch
    sample, _ = sample_queries(queries, sample_size)
    key = _key(db, sample, gap_open, gap_extend)
    if cache:
        with _lock:
            hit = _load(cache).get(key)
        if hit:
            return {"options": hit["options"], "timings": hit.get("timings", []), "key": key,
                    "cached": True}
    cands = cands or candidates(db)
    q = torch.from_numpy(sample.res).cuda(db.device)
    ql = torch.from_numpy(sample.lens).cuda(db.device)
    out = torch.empty((len(sample), db.n), dtype=torch.int32, device=f"cuda:{db.device}")
    timings = []
    for opt in cands:
        try:
            plan = db.plan(len(sample), max(sample.total, 1), **opt)
        except swgb.SwError:
            continue  # e.g. a shape that cannot launch on this device
        plan.search(q, ql, gap_open, gap_extend, out=out)  # warm-up (graph capture)
        best = float("inf")
        for _ in range(repeats):
            plan.search(q, ql, gap_open, gap_extend, out=out)
            st = plan.stats()
            # the whole search: the cutoff moves work between the kernels
            best = min(best, st["pair_ms"] + st["search_ms"] + st["recompute_ms"])
        plan.close()
        timings.append((opt, best))
    if not timings:
        raise RuntimeError("no candidate tile shape could run")
    best_opt = min(timings, key=lambda t: t[1])[0]
    if cache:
        with _lock:
            os.makedirs(os.path.dirname(cache), exist_ok=True)
            data = _load(cache)
            data[key] = {"options": best_opt, "timings": timings}
            tmp = cache + f".tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(data, fh, indent=1)
            os.replace(tmp, cache)
    return {"options": best_opt, "timings": timings, "key": key, "cached": False}
