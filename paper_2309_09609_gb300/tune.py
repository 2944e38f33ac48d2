"""Autotuner for the search plan's tile shape.

The options (all of which change speed only, never a score):

* two queries per word in the inter-task kernel (``two_query``: by the
  plan's cost model, or never); its strip height stays at 32 rows, the only
  height compiled with the gap penalties as constants (on the batched
  workload a tuner that tried 24 rows on its 8-query sample picked them, and
  the full batch then ran 7% slower);
* the one-query inter-task kernel's rows per thread (32, 16), columns per
  wavefront with 32 rows (8, 4) and warps per block (8, 4);
* the inter/intra length cutoff (1500, 3000, 7000, none) and the rows per
  lane of the int32 intra-task kernel (8, 16).

The search is a coordinate descent from the defaults: for each option in
turn every alternative value is timed with the others at their best so far,
and the best is kept; a second pass repeats this, and stops early once a
pass changes nothing.  No option set is timed twice.  On the batched-uneven
workload that is 15-20 searches of the sample instead of the 90 of the full
product.  Each candidate runs a plan over a length-stratified sample of the
batch's queries against the whole resident database and is timed by the
plan's own CUDA events around all of its kernels (pair, inter-task and
recompute).  The best is cached in a JSON file keyed by GPU, SM count,
database signature, the sample's query length profile and the gap penalties.

One shape serves the whole batch: the search is one persistent launch per
kernel over every (query, subject-group) item, so its kernels run one
configuration.  What does differ per length bucket is decided per item by
the plan itself: which subjects go to the pair kernels (the cutoff), which
pair-kernel width a query takes, and how queries are dealt to query
streams.
"""
from __future__ import annotations

import json
import os
import threading

import numpy as np

from . import swgb

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "swgb", "tune.json")
NO_CUTOFF = 1 << 30
_lock = threading.Lock()


def space(db, n_queries: int) -> dict:
    """The values of each option, defaults first.  Cutoffs at or above the
    longest subject collapse into "none"; the int32 row count matters only
    when some cutoff sends subjects to the pair kernels (for their saturated
    pairs); the two-query options only with two or more queries."""
    maxlen = db.max_length
    cuts = []
    for c in (1500, 3000, 7000, NO_CUTOFF):
        c = c if c < maxlen else NO_CUTOFF
        if c not in cuts:
            cuts.append(c)
    sp = {}
    if n_queries >= 2:
        sp["two_query"] = [1, 0]
    sp["rows_per_thread"] = [32, 16]
    sp["inter_columns"] = [8, 4]
    sp["warps_per_block"] = [8, 4]
    sp["long_cutoff"] = cuts
    if cuts[0] < maxlen:
        sp["intra_rows"] = [8, 16]
    return sp


def valid(opt: dict) -> bool:
    """Eight columns per wavefront need 32 rows per thread."""
    return not (opt.get("rows_per_thread") == 16 and opt.get("inter_columns") == 8)


def descend(sp: dict, measure, passes: int = 2):
    """Coordinate descent over the option space `sp` (option -> values,
    default first): returns (best options, [(options, cost), ...] in the
    order timed).  `measure(options)` gives a cost, or None when the option
    set cannot run; invalid sets are skipped and none is measured twice."""
    seen = {}
    order = []

    def cost(opt):
        key = tuple(sorted(opt.items()))
        if key not in seen:
            c = measure(dict(opt)) if valid(opt) else None
            seen[key] = c
            if c is not None:
                order.append((dict(opt), c))
        return seen[key]

    best = {k: v[0] for k, v in sp.items()}
    if not valid(best):
        best["inter_columns"] = 4
    best_cost = cost(best)
    if best_cost is None:
        raise RuntimeError("the default tile shape cannot run")
    for _ in range(passes):
        changed = False
        for name, values in sp.items():
            for v in values:
                if v == best[name]:
                    continue
                trial = dict(best, **{name: v})
                c = cost(trial)
                if c is not None and c < best_cost:
                    best, best_cost, changed = trial, c, True
        if not changed:
            break
    return best, order


def sample_queries(queries, k: int = 8):
    """Up to k queries at evenly spaced length quantiles of the batch."""
    n = len(queries)
    if n <= k:
        return queries, np.arange(n)
    order = np.argsort(queries.lens, kind="stable")
    idx = order[np.unique(np.linspace(0, n - 1, k).round().astype(int))]
    return queries.subset(idx), idx


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
         repeats: int = 2, cache: str | None = DEFAULT_CACHE, sample_size: int = 8,
         passes: int = 2):
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
    q = torch.from_numpy(sample.res).cuda(db.device)
    ql = torch.from_numpy(sample.lens).cuda(db.device)
    out = torch.empty((len(sample), db.n), dtype=torch.int32, device=f"cuda:{db.device}")

    def measure(opt):
        try:
            plan = db.plan(len(sample), max(sample.total, 1), **opt)
        except swgb.SwError:
            return None  # e.g. a shape that cannot launch on this device
        plan.search(q, ql, gap_open, gap_extend, out=out)  # warm-up (graph capture)
        best = float("inf")
        for _ in range(repeats):
            plan.search(q, ql, gap_open, gap_extend, out=out)
            st = plan.stats()
            # the whole search: the cutoff moves work between the kernels
            best = min(best, st["pair_ms"] + st["search_ms"] + st["recompute_ms"])
        plan.close()
        return best

    best_opt, timings = descend(space(db, len(sample)), measure, passes)
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
