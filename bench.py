"""Benchmark: exact Smith-Waterman/Gotoh protein database search on GB300.

Workload (default): 20 queries of 144-5478 residues (log-spaced) against a
synthetic database of 570,000 subjects with lognormal lengths (mean 360,
~205 M residues), BLOSUM62, gap open 10 / extend 2 -- the shape of the
paper's search (Section IV-A), synthetic because Env-NR is not available.

One step = one exact search of all queries against the whole database
through a plan: the packed pair kernel (long subjects), the packed inter-task
kernel (the rest) and the int32 intra-task kernel (saturated pairs), replayed
from a CUDA graph.  Printed: one JSON line with GCUPS (cells = sum of query
lengths x sum of subject lengths), per-step latency p50/p99, the plain int32
one-query-per-launch baseline, the integer roofline of the dominant kernel
against the intpeak microbenchmark, the end-to-end rate through the C ABI
with host buffers, and the CPU oracle timed on a bounded sample on the host
cores.

Under torchrun (``--gpus N``) each rank searches its own seeded instance of
the workload (seed + rank) on its GPU; the printed value is the cells of all
ranks over the longest rank's timed region (weak scaling).

``--impl reference`` times the CPU oracle instead (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GCUPS on 1 GB300 (batched packed vs plain int32), bit-exact scores; p50/p99 latency"
WORKLOADS = ("paper-search", "plain-small", "batched-uneven", "long")

# CPU oracle sample budgets (cells): the baseline leg, and one reference-arm
# step.  On 16 Arm cores the oracle scored the long-sequence pairs at
# 0.5-0.8 GCUPS and the short-subject workloads at 8.3-8.5, hence the smaller
# budget.
CPU_CELLS = {"paper-search": 1e11, "batched-uneven": 1e11, "plain-small": 1e11, "long": 1e10}
REF_CELLS = {"paper-search": 1.5e10, "batched-uneven": 1.5e10, "plain-small": 1.5e10, "long": 2e9}

# algorithmic ALU-pipe lane-operations per cell of the packed recurrence: per
# 32-bit word (2 cells) one prmt (profile pair), vimax3 (E', F', Go), viaddmax
# (H'), viaddmax (E' next column), viaddmax (F' next row) and half a vimax3 (S);
# H' - Go is an IMAD on the FMA pipe and is not counted
PACKED_ALU_OPS_PER_CELL = 5.5 / 2
# the same with two queries per word: the profile word is read ready-made,
# so the prmt drops out (4.5 per word)
TWO_QUERY_ALU_OPS_PER_CELL = 4.5 / 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="paper-search", choices=WORKLOADS)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--rows", type=int, default=None, help="packed rows per thread (16/32)")
    ap.add_argument("--cutoff", type=int, default=None, help="inter/intra length cutoff")
    ap.add_argument("--overlap", type=int, default=None, choices=[0, 1],
                    help="plan option overlap_kernels (inter-task kernels beside the pair kernels)")
    ap.add_argument("--auto-cutoff", type=int, default=None, choices=[0, 1],
                    help="plan option auto_cutoff (load balance of few-query searches)")
    ap.add_argument("--warps", type=int, default=None)
    ap.add_argument("--cols", type=int, default=None, help="inter-task wavefront columns (4/8)")
    ap.add_argument("--two-query", type=int, default=None, choices=[0, 1, 2],
                    help="two queries per word in the inter-task kernel: 0 never, 1 auto, 2 always")
    ap.add_argument("--two-query-rows", type=int, default=None, choices=[16, 24, 32])
    ap.add_argument("--two-query-pairs", type=int, default=None,
                    help="stream pairs of the two-query kernels (default: the plan's choice)")
    ap.add_argument("--two-query-long", type=int, default=None, choices=[0, 1, 2],
                    help="two queries per word against long subjects: 0 never, 1 auto, 2 always")
    ap.add_argument("--wide-min", type=int, default=None,
                    help="shortest query scored 32 rows per lane against long subjects")
    ap.add_argument("--wide-min-subject", type=int, default=None,
                    help="shortest subject pair scored 32 rows per lane")
    ap.add_argument("--cpu-cells", type=float, default=None,
                    help="cell budget of the CPU oracle baseline's sample (all queries x the "
                         "first subjects that fit); default per workload, 10-30 s on 16 cores")
    ap.add_argument("--ref-cells", type=float, default=None,
                    help="cell budget of one reference-arm step (the CPU oracle); default per "
                         "workload, a few seconds")
    ap.add_argument("--subjects", type=int, default=None,
                    help="shrink the database (profiling / small cases)")
    ap.add_argument("--queries", type=int, default=None, help="keep only N queries")
    ap.add_argument("--query-offset", type=int, default=0, help="first query kept by --queries")
    ap.add_argument("--serve", type=int, default=1000,
                    help="serving leg: arrivals replayed against the resident DB (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=50.0, help="Poisson arrival rate (1/s)")
    ap.add_argument("--serve-slots", type=int, default=2,
                    help="concurrent batches (plans with their own stream) in the serving leg")
    ap.add_argument("--serve-batch", type=int, default=16, help="largest batch of the serving leg")
    ap.add_argument("--tune", action="store_true",
                    help="pick the tile shape with the autotuner before timing")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the plan's kernels directly instead of replaying a CUDA graph "
                         "(for kernel profilers)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-align", action="store_true", help="skip the traceback leg")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-shard", action="store_true",
                    help="under several ranks, skip the one-search-over-all-ranks leg")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the batched-uneven and long-sequence records of the default run")
    ap.add_argument("--config-steps", type=int, default=2,
                    help="timed steps of each further workload record (about 6-9 s each)")
    return ap.parse_args()


L2_BYTES = 129 * 10 ** 6


def l2_flush_bytes(db_residues: int) -> int:
    """Bytes to write between timed steps so that none starts with the
    database in L2: 0 when its two device layouts (about 2 bytes per
    residue, both read) already exceed the 129 MB L2, else twice the L2."""
    return 0 if 2 * db_residues > L2_BYTES else 2 * L2_BYTES


def l2_note(db_residues: int) -> str:
    """How the timed region stands to the 129 MB L2."""
    if not l2_flush_bytes(db_residues):
        return (f"no flush: device-resident DB layouts (~{2 * db_residues / 1e6:.0f} MB) "
                f"> 129 MB L2")
    return (f"L2 flushed between timed steps: DB layouts (~{2 * db_residues / 1e6:.1f} MB) "
            f"fit in L2, so a {2 * L2_BYTES / 1e6:.0f} MB buffer is written after each step, "
            f"outside its CUDA events")


def paper_arch_efficiency(gcups_per_gpu, i32_rate, sms, mhz) -> dict:
    """The paper's architectural efficiency (Section II-C, Eq. 4-5): achieved
    GCUPS over the peak of Algorithm 1's 12 int32 instructions per cell at
    the measured int32 max rate (lane-ops per SM clock x SMs x clock; one
    ALU-pipe instruction, which the algorithm's six max operations need).
    The packed path does two cells per 5.5 ALU ops, so it can exceed 1."""
    from paper_2309_09609_gb300 import perfmodel
    peak = perfmodel.theoretical_peak_gcups(sms, 1, i32_rate, mhz)
    return {"value": round(perfmodel.arch_efficiency(gcups_per_gpu, peak), 4),
            "peak_gcups": round(peak, 1),
            "model": f"Eq. 5: imax {i32_rate:.1f} lane-ops/clk/SM x {sms} SMs x {mhz:.0f} MHz "
                     f"/ {perfmodel.PAPER_INSTRUCTIONS_PER_CELL} instructions per cell"}


def workload_config(w) -> dict:
    """The keys that name a workload in both arms' config."""
    return {"workload": w.name, "queries": len(w.queries), "subjects": len(w.db),
            "query_residues": w.queries.total, "db_residues": w.db.total, "cells": w.cells,
            "gaps": [w.gap_open, w.gap_extend], "matrix": "BLOSUM62",
            "planted_homologs": int(w.planted.size)}


def rank_workload(args, rank):
    """The workload one rank searches: with several ranks, each takes its own
    seeded instance of the same shape (seed + rank: its own queries and
    database partition), so the ranks shard independent searches and need no
    collective on the data path (weak scaling).  Rank 0 searches exactly the
    one-GPU workload."""
    return make_workload(args.workload, args.seed + rank, args.subjects, args.queries,
                         args.query_offset)


def make_workload(name, seed, subjects=None, queries=None, query_offset=0):
    from paper_2309_09609_gb300 import synth
    kw = {}
    if subjects and name in ("paper-search", "batched-uneven", "long"):
        kw["n_subjects"] = subjects
    w = {"paper-search": synth.paper_search, "plain-small": synth.plain_small,
         "batched-uneven": synth.batched_uneven, "long": synth.long_sequences}[name](seed, **kw)
    if queries and queries + query_offset <= len(w.queries) and queries < len(w.queries):
        w.queries = w.queries.subset(range(query_offset, query_offset + queries))
        w.name += f" (queries {query_offset}..{query_offset + queries - 1})"
    return w


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device=0):
        self.device = device
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.file:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.file.flush()
        rows = []
        with open(self.file.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(power) if power else None}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("SWGB_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
        return rank, world, local, dist
    return rank, world, local, None


def _reduce_over_ranks(x, dist, device, op):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64,
                     device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (a scalar: the timed region's length)."""
    return _reduce_over_ranks(x, dist, device, None if dist is None else dist.ReduceOp.MAX)


def sum_over_ranks(x, dist, device):
    """The sum of x over all ranks (a scalar: the cells every rank scored)."""
    return _reduce_over_ranks(x, dist, device, None if dist is None else dist.ReduceOp.SUM)


def oracle_sample(w, cell_budget):
    """All queries vs the longest prefix of subjects (by caller index, which is
    random with respect to length) whose cells fit `cell_budget`; at least one."""
    per = np.cumsum(w.db.lens.astype(np.int64)) * int(w.queries.total)
    n = max(1, int(np.searchsorted(per, cell_budget, side="right")))
    return w.db.subset(np.arange(n))


def time_oracle(w, sub, nthreads):
    import oracle
    nq, nd = len(w.queries), len(sub)
    pq = np.repeat(np.arange(nq, dtype=np.int32), nd)
    pd = np.tile(np.arange(nd, dtype=np.int64), nq)
    t0 = time.perf_counter()
    s = oracle.pairs_packed(w.queries.res, w.queries.offs, w.queries.lens, sub.res, sub.offs,
                            sub.lens, pq, pd, w.gap_open, w.gap_extend, None, nthreads)
    dt = time.perf_counter() - t0
    cells = w.queries.total * sub.total
    return s.reshape(nq, nd), cells, dt


def run_reference(args):
    """Reference arm: the CPU oracle, as it stands, on the host cores."""
    rank, world, local, dist = dist_setup(args)
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = make_workload(args.workload, args.seed, args.subjects, args.queries, args.query_offset)
    sub = oracle_sample(w, args.ref_cells or REF_CELLS[args.workload])
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        time_oracle(w, sub, cores)
    times = []
    for _ in range(args.steps):
        _, cells, dt = time_oracle(w, sub, cores)
        times.append(dt)
    ms = 1e3 * statistics.mean(times)
    g = cells / (ms / 1e3) / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": round(g, 4), "unit": "GCUPS",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
           "data": "synthetic",
           "config": {**workload_config(w), "parallelism": f"{cores} host threads",
                      "sample": f"all {len(w.queries)} queries x first {len(sub)} subjects "
                      f"({cells:.3e} cells per step)"},
           "cpu_baseline": {"value": round(g, 4), "unit": "GCUPS", "cores": cores,
                            "kind": "oracle", "sample": f"{len(sub)} subjects x all queries"},
           "e2e": {"value": round(g, 4), "unit": "GCUPS", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


CSRC = os.path.join(ROOT, "paper_2309_09609_gb300", "csrc")
# ncu DRAM records of a dominant kernel on a benchmark workload, each valid
# while the kernel's own sources hash to the recorded value:
# (kernel, workload) -> (record file, sources hashed in order)
TRAFFIC_RECORDS = {
    ("inter2q_kernel", "paper-search"): ("inter2q_kernel_paper-search_traffic.txt",
                                         ("inter2q_kernel.cu", "device_common.cuh")),
    ("pair2q_kernel", "long"): ("pair2q_kernel_long-sequences_traffic.txt",
                                ("pair2q_kernel.cu", "device_common.cuh")),
}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", TRAFFIC_RECORDS[("inter2q_kernel", "paper-search")][0])
KERNEL_SOURCES = [os.path.join(CSRC, f) for f in TRAFFIC_RECORDS[("inter2q_kernel", "paper-search")][1]]


def kernel_sources_sha256(sources=None):
    import hashlib
    h = hashlib.sha256()
    for f in sources or KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_record(path=None):
    rec = {}
    path = path or TRAFFIC_FILE
    if os.path.exists(path):
        with open(path) as fh:
            for line in fh:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    rec[k.strip()] = v.strip()
    return rec


def profiled_traffic(args, kernel="inter2q_kernel"):
    """DRAM bytes per launch of the dominant kernel from its committed ncu
    record, if the record covers this workload at its default size and plan,
    and the kernel's sources are unchanged since the capture."""
    key = (kernel, args.workload)
    if key not in TRAFFIC_RECORDS:
        return None
    default = (not args.subjects and not args.queries and args.rows in (None, 32)
               and args.warps in (None, 8) and args.cutoff in (None, 1500) and not args.tune
               and getattr(args, "cols", None) in (None, 8)
               and getattr(args, "two_query", None) is None
               and getattr(args, "two_query_rows", None) is None
               and getattr(args, "two_query_pairs", None) is None
               and getattr(args, "two_query_long", None) is None
               and getattr(args, "auto_cutoff", None) is None
               and getattr(args, "overlap", None) is None
               and getattr(args, "wide_min", None) is None
               and getattr(args, "wide_min_subject", None) is None)
    fname, srcs = TRAFFIC_RECORDS[key]
    rec = traffic_record(os.path.join(ROOT, "profiles", fname))
    sha = kernel_sources_sha256([os.path.join(CSRC, f) for f in srcs])
    if not default or rec.get("kernel_sources_sha256") != sha:
        return None
    return int(rec["dram_bytes_per_launch"])


def run_serving(d, db, args, opts, w):
    """Replays a Poisson trace (lognormal query lengths, mean 400) against the
    resident database through the continuous-batching server."""
    from paper_2309_09609_gb300 import serve, synth
    trace = synth.serving_trace(seed=args.seed, n=args.serve, rate=args.serve_rate)
    srv = serve.Server(d, slots=args.serve_slots, max_batch=args.serve_batch,
                       max_batch_residues=max(65536, 4096 * args.serve_batch),
                       gap_open=w.gap_open, gap_extend=w.gap_extend, **opts)
    t0 = time.perf_counter()
    try:
        futs = serve.replay(srv, trace)
    finally:
        srv.close()
    wall = time.perf_counter() - t0
    rep = srv.report(wall)
    # a few requests recomputed alone must equal their rows from the mix
    check = np.linspace(0, len(trace.queries) - 1, 4).astype(int)
    same = all((d.search(trace.queries.seq(int(i)), np.array([trace.queries.lens[i]], np.int32),
                         w.gap_open, w.gap_extend)[0] == futs[int(i)].result()).all() for i in check)
    offered = args.serve_rate * float(trace.queries.lens.mean()) * db.total / 1e9
    return {"arrivals": len(trace.queries), "rate_per_s": args.serve_rate,
            "p50_ms": round(rep["p50_ms"], 2), "p99_ms": round(rep["p99_ms"], 2),
            "gcups": round(rep["gcups"], 1), "offered_gcups": round(offered, 1),
            "batches": rep["batches"], "mean_batch": round(rep["mean_batch"], 2),
            "max_concurrent_batches": rep["max_concurrent_batches"], "slots": args.serve_slots,
            "max_batch": args.serve_batch,
            "wall_s": round(wall, 2), "alone_equals_mixed": bool(same)}


def run_align(d, q, db, scores, w):
    """Optimal alignments (with traceback) of every query's best-scoring
    subject; the call is timed with the host clock around sw_align, which is
    synchronous and includes its allocations and copies."""
    import oracle
    best = scores.argmax(dim=1).cpu().numpy() if hasattr(scores, "argmax") else scores.argmax(1)
    pq = np.arange(len(q), dtype=np.int32)
    ps = best.astype(np.int64)
    d.align(q.res, q.lens, pq[:1], ps[:1], w.gap_open, w.gap_extend)      # warm-up
    t0 = time.perf_counter()
    got = d.align(q.res, q.lens, pq, ps, w.gap_open, w.gap_extend)
    ms = 1e3 * (time.perf_counter() - t0)
    cells = int(sum(int(q.lens[a]) * int(db.lens[b]) for a, b in zip(pq, ps)))
    oracle.build()
    same = all(got[k] == oracle.align(q.seq(int(a)), db.seq(int(b)), w.gap_open, w.gap_extend)
               for k, (a, b) in enumerate(zip(pq, ps)))
    return {"pairs": int(pq.size), "cells": cells, "ms": round(ms, 3),
            "gcups": round(cells / (ms / 1e3) / 1e9, 2),
            "transcript_columns": int(sum(len(g["ops"]) for g in got)),
            "equals_oracle": bool(same)}


def timed_steps(plan, q_dev, l_dev, out, w, steps, warmup, stream, local, dist):
    """W untimed warm-up searches, then exactly `steps` timed ones between a
    barrier and synchronize on both sides, with CUDA events on the plan's
    stream and nvidia-smi clocks sampled meanwhile.  When the database fits
    in L2, a buffer of twice its size is written after each step, between
    that step's end event and the next one's start, and the total is the
    sum of the steps."""
    import torch

    def step():
        plan.search(q_dev, l_dev, w.gap_open, w.gap_extend, None, out=out, stream=stream)

    flush = l2_flush_bytes(int(w.db.total))
    scratch = torch.empty(flush // 4, dtype=torch.int32, device=out.device) if flush else None
    for _ in range(max(warmup, 1)):
        step()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = starts[1:] + [torch.cuda.Event(enable_timing=True)]
    if flush:
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    kernel_ms, recompute_ms, pair_ms = [], [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(steps):
            if flush or i == 0:
                starts[i].record(stream)
            step()
            ends[i].record(stream)
            if flush:
                with torch.cuda.stream(stream):
                    scratch.fill_(i)
            st = plan.stats()
            kernel_ms.append(st["search_ms"])
            recompute_ms.append(st["recompute_ms"])
            pair_ms.append(st["pair_ms"])
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [starts[i].elapsed_time(ends[i]) for i in range(steps)]
    total_ms = sum(step_ms) if flush else starts[0].elapsed_time(ends[-1])
    return {"step_ms": step_ms, "total_ms": total_ms, "kernel_ms": kernel_ms,
            "recompute_ms": recompute_ms, "pair_ms": pair_ms, "stats": plan.stats(),
            "clocks": clk.summary(), "l2_flush_bytes": flush}


def roofline(t, peak, peak_source, rate_mhz, traffic):
    """The integer roofline of the dominant kernel of a timed search: ALU-pipe
    lane-ops vs the intpeak microbenchmark's measured DPX throughput (SMs x
    clock x per-SM rate).  The inter-task kernel scores the short subjects'
    cells, the packed pair kernel the rest (subjects longer than the cutoff);
    both run the same packed recurrence, so both count the same lane-ops per
    cell."""
    stats = t["stats"]
    per_kernel = {}
    two_q = stats.get("inter2_items", 0) > 0
    two_q_long = stats.get("pair2_items", 0) > 0
    inter_name = ("inter2q_kernel (packed inter-task, two queries per word)" if two_q
                  else "inter_kernel (packed inter-task)")
    pair_name = ("pair2q_kernel (packed intra-task, two queries per word)" if two_q_long
                 else "pair_kernel (packed intra-task)")
    for name, kcells, kms_list, ops in (
            (inter_name, stats["inter_cells"], t["kernel_ms"],
             TWO_QUERY_ALU_OPS_PER_CELL if two_q else PACKED_ALU_OPS_PER_CELL),
            (pair_name, stats["cells"] - stats["inter_cells"], t["pair_ms"],
             TWO_QUERY_ALU_OPS_PER_CELL if two_q_long else PACKED_ALU_OPS_PER_CELL)):
        kms = statistics.mean(kms_list) if kms_list else float("nan")
        ach = ops * kcells / (kms / 1e3) / 1e12 if kcells else 0.0
        per_kernel[name] = {"ms": round(kms, 3), "cells": int(kcells), "achieved": round(ach, 3),
                            "frac": round(ach / peak, 4), "alu_ops_per_cell": ops}
    dominant = max(per_kernel, key=lambda k: per_kernel[k]["ms"])
    dom = per_kernel[dominant]
    inter = dominant.startswith("inter")
    return {"bound": "alu", "achieved": dom["achieved"], "peak": round(peak, 3),
            "unit": "Tops/s", "frac": dom["frac"],
            "traffic": traffic(("inter2q_kernel" if two_q else "inter_kernel") if inter
                               else ("pair2q_kernel" if two_q_long else "pair_kernel")),
            "kernel": dominant, "kernel_ms": dom["ms"], "kernel_cells": dom["cells"],
            "kernels": per_kernel,
            "alu_ops_per_cell": dom["alu_ops_per_cell"],
            "peak_source": peak_source,
            "intpeak_clock_mhz": round(rate_mhz, 1),
            "peak_gcups": round(peak * 1e12 / dom["alu_ops_per_cell"] / 1e9, 1),
            "pair_kernel_ms": per_kernel[pair_name]["ms"],
            "recompute_ms": round(statistics.mean(t["recompute_ms"]), 3)}


def cpu_leg(w, got_host, budget):
    """The CPU oracle on all queries x the first subjects that fit `budget`
    cells, on every host core: the baseline, and parity of those pairs."""
    import oracle
    oracle.build()
    sub = oracle_sample(w, budget)
    cores = os.cpu_count() or 1
    ref, ocells, odt = time_oracle(w, sub, cores)
    got = np.asarray(got_host)[:, :len(sub)]
    return ({"value": round(ocells / odt / 1e9, 4), "unit": "GCUPS", "cores": cores,
             "kind": "oracle",
             "sample": f"all {len(w.queries)} queries x first {len(sub)} subjects "
                       f"({ocells:.3e} cells, {odt:.1f} s)"},
            bool((got == ref).all()))


def plain_leg(d, q, w, device, stream, rows=None):
    """The plain int32 one-query-per-launch baseline (sw_search_plain) on the
    queries `rows` (default all), timed with CUDA events; and its scores."""
    import torch
    sub = q if rows is None else q.subset(rows)
    qd = torch.from_numpy(sub.res).to(device)
    ld = torch.from_numpy(sub.lens).to(device)
    outp = torch.empty((len(sub), d.n), dtype=torch.int32, device=device)
    d.search_plain(qd, ld, w.gap_open, w.gap_extend, out=outp, stream=stream)  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    d.search_plain(qd, ld, w.gap_open, w.gap_extend, out=outp, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    pms = e0.elapsed_time(e1)
    cells = sub.total * w.db.total
    return {"value": round(cells / (pms / 1e3) / 1e9, 2), "unit": "GCUPS", "ms": round(pms, 3),
            "launches": len(sub)}, outp


def e2e_leg(plan, q, N, w, repeats, dist, device):
    """The search through the C ABI with host (pinned) buffers, the query
    upload and the score download inside the timed region."""
    import torch
    q_host = torch.from_numpy(q.res).pin_memory()
    l_host = torch.from_numpy(q.lens).pin_memory()
    out_host = torch.empty((len(q), N), dtype=torch.int32).pin_memory()
    plan.search(q_host, l_host, w.gap_open, w.gap_extend, None, out=out_host)
    e2e = []
    for _ in range(max(1, repeats)):
        t0 = time.perf_counter()
        plan.search(q_host, l_host, w.gap_open, w.gap_extend, None, out=out_host)
        e2e.append(time.perf_counter() - t0)
    return max_over_ranks(statistics.mean(e2e), dist, device), out_host


def run_config(name, args, device, local, stream, peak, peak_src, rate_mhz):
    """A further workload measured in the same run (one GPU): its own timed
    steps, roofline, plain-baseline speed-up, e2e, CPU baseline and parity
    on the CPU sample."""
    import torch
    from paper_2309_09609_gb300 import swgb
    w = make_workload(name, args.seed)
    q, db = w.queries, w.db
    d = swgb.Database.from_seqset(db, device=local)
    opts, tuned = {}, None
    if name == "batched-uneven":    # the autotuned plan, replayed from one graph
        from paper_2309_09609_gb300 import tune
        t0 = time.perf_counter()
        tr = tune.tune(d, q, w.gap_open, w.gap_extend, cache=None)
        opts = dict(tr["options"], use_graph=1)
        tuned = {"options": tr["options"], "candidates": len(tr["timings"]),
                 "seconds": round(time.perf_counter() - t0, 2)}
    plan = d.plan(len(q), q.total, **opts)
    q_dev = torch.from_numpy(q.res).to(device)
    l_dev = torch.from_numpy(q.lens).to(device)
    out = torch.empty((len(q), len(db)), dtype=torch.int32, device=device)
    steps = args.config_steps
    t = timed_steps(plan, q_dev, l_dev, out, w, steps, args.warmup, stream, local, None)
    ms = t["total_ms"] / steps
    rec = {"workload": workload_config(w), "value": round(w.cells / (ms / 1e3) / 1e9, 2),
           "unit": "GCUPS", "steps": steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
           "latency_ms": {"p50": round(float(np.percentile(t["step_ms"], 50)), 3),
                          "p99": round(float(np.percentile(t["step_ms"], 99)), 3)},
           "l2": l2_note(db.total), "recomputed_pairs": t["stats"]["recomputed_pairs"],
           "gpu_launches": t["stats"]["kernels_launched"] * steps,
           "plan": {k: getattr(swgb.options(**opts), k) for k, _ in swgb.Options._fields_},
           "autotuned": tuned, "clocks": t["clocks"]}
    sub_args = argparse.Namespace(**{**vars(args), "workload": name, "tune": name == "batched-uneven"})
    rec["roofline"] = roofline(t, peak, peak_src, rate_mhz, lambda k: profiled_traffic(sub_args, k))
    # plain int32 baseline: one launch per query, so its rate per query does
    # not depend on how many queries run; timed on a stated sample
    if name == "batched-uneven":
        rows = np.arange(0, len(q), 20)
        pl, outp = plain_leg(d, q, w, device, stream, rows)
        pl["sample"] = f"{rows.size} of {len(q)} queries (every 20th), all subjects"
        rec["plain_int32"] = pl
        rec["plain_equals_packed"] = bool(torch.equal(outp, out[torch.from_numpy(rows).to(device)]))
    else:
        # long subjects: the plain kernel gives each subject one thread, so a
        # launch lasts as long as its longest pair (about 16 s for the
        # shortest query here, minutes for all eight).  Timed on the shortest
        # query against every subject: the same threads and the same spread
        # of their work as a launch of any other query, so the same rate (a
        # subset of short subjects would leave most of the GPU idle and
        # understate the baseline: 52 GCUPS on 2,000 subjects of at most
        # 8,000 residues, against 241 for all eight queries and subjects)
        qi = int(np.argmin(q.lens))
        pl, outp = plain_leg(d, q, w, device, stream, [qi])
        pl["sample"] = f"the shortest query ({int(q.lens[qi])} residues) x all {len(db)} subjects"
        rec["plain_int32"] = pl
        rec["plain_equals_packed"] = bool(torch.equal(outp[0], out[qi]))
    rec["speedup_vs_plain"] = round(rec["value"] / pl["value"], 3)
    e2e_s, out_host = e2e_leg(plan, q, len(db), w, 1, None, device)
    rec["e2e"] = {"value": round(w.cells / e2e_s / 1e9, 2), "unit": "GCUPS",
                  "h2d_bytes_per_step": int(q.total + 4 * len(q)),
                  "d2h_bytes_per_step": int(4 * len(q) * len(db)),
                  "ms_per_step": round(1e3 * e2e_s, 3)}
    if not args.no_cpu:
        rec["cpu_baseline"], rec["parity_on_cpu_sample"] = cpu_leg(
            w, out_host.numpy(), CPU_CELLS[name])
    plan.close()
    d.close()
    return rec


def run_sharded(args, rank, world, local, device, dist, one_gpu_scores):
    """The one-GPU workload (seed, not seed + rank) as ONE search over all
    ranks: each rank scores its cell-weighted partition of the database, and
    the int32 columns are all-gathered in caller order.  Timed between
    barriers, all-gather included, max over ranks.  Rank 0 checks the
    gathered matrix against its own one-GPU search of the same workload."""
    import torch
    from paper_2309_09609_gb300 import shard
    w = make_workload(args.workload, args.seed, args.subjects, args.queries, args.query_offset)
    sd = shard.ShardedDatabase(w.db, dist, device=local)
    sd.search(w.queries.res, w.queries.lens, w.gap_open, w.gap_extend)      # warm-up
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        got = sd.search(w.queries.res, w.queries.lens, w.gap_open, w.gap_extend)
    torch.cuda.synchronize()
    dist.barrier()
    ms = max_over_ranks(1e3 * (time.perf_counter() - t0) / args.steps, dist, device)
    rec = {"value": round(w.cells / (ms / 1e3) / 1e9, 2), "unit": "GCUPS",
           "ms_per_step": round(ms, 3), "scaling": "strong", "steps": args.steps,
           "subjects_per_rank": sd.sizes.tolist(),
           "residues_per_rank": [int(w.db.lens[sd.bounds[r]:sd.bounds[r + 1]].sum())
                                 for r in range(world)],
           "note": "host clock around search + all-gather of the int32 columns (host buffers)"}
    if one_gpu_scores is not None:
        rec["equals_one_gpu"] = bool((one_gpu_scores.cpu().numpy() == got).all())
    return rec


def run_native(args):
    import torch
    rank, world, local, dist = dist_setup(args)
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2309_09609_gb300 import swgb

    w = rank_workload(args, rank)
    q, db = w.queries, w.db
    nq, N = len(q), len(db)
    cells = w.cells
    t0 = time.perf_counter()
    d = swgb.Database.from_seqset(db, device=local)
    db_create_s = time.perf_counter() - t0
    opts = {}
    if args.rows:
        opts["rows_per_thread"] = args.rows
    if args.cutoff is not None:
        opts["long_cutoff"] = args.cutoff
    if args.auto_cutoff is not None:
        opts["auto_cutoff"] = args.auto_cutoff
    if args.overlap is not None:
        opts["overlap_kernels"] = args.overlap
    if args.warps:
        opts["warps_per_block"] = args.warps
    if args.cols:
        opts["inter_columns"] = args.cols
    if args.no_graph:
        opts["use_graph"] = 0
    if args.two_query is not None:
        opts["two_query"] = args.two_query
    if args.two_query_rows is not None:
        opts["two_query_rows"] = args.two_query_rows
    if args.two_query_pairs is not None:
        opts["two_query_pairs"] = args.two_query_pairs
    if args.two_query_long is not None:
        opts["two_query_long"] = args.two_query_long
    if args.wide_min is not None:
        opts["wide_min_len"] = args.wide_min
    if args.wide_min_subject is not None:
        opts["wide_min_subject"] = args.wide_min_subject
    tuned = None
    if args.tune:
        from paper_2309_09609_gb300 import tune
        t0 = time.perf_counter()
        tuned = tune.tune(d, q, w.gap_open, w.gap_extend, cache=None)
        opts.update(tuned["options"])
        tuned = {"options": tuned["options"], "candidates": len(tuned["timings"]),
                 "seconds": round(time.perf_counter() - t0, 2)}
    plan = d.plan(nq, q.total, **opts)
    stream = torch.cuda.Stream(device=device)
    q_dev = torch.from_numpy(q.res).to(device)
    l_dev = torch.from_numpy(q.lens).to(device)
    out = torch.empty((nq, N), dtype=torch.int32, device=device)

    # timed region: device-resident inputs (the DB layouts, ~2 x residues bytes,
    # exceed the 129 MB L2, so no flush is needed between steps)
    t = timed_steps(plan, q_dev, l_dev, out, w, args.steps, args.warmup, stream, local, dist)
    total_ms = max_over_ranks(t["total_ms"], dist, device)
    ms = total_ms / args.steps
    all_cells = sum_over_ranks(float(cells), dist, device)   # each rank its own search
    gcups = all_cells / (ms / 1e3) / 1e9
    stats = t["stats"]
    clocks = t["clocks"]

    result = {"metric": METRIC, "value": round(gcups, 2), "unit": "GCUPS", "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
              "dtype": "i16x2+i32", "data": "synthetic",
              "config": {**workload_config(w),
                         "l2": l2_note(db.total),
                         "parallelism": (f"{world} GPUs, one independent search each "
                                         f"(seed + rank)") if world > 1 else "1 GPU",
                         "plan": {k: getattr(swgb.options(**opts), k) for k, _ in swgb.Options._fields_}},
              "latency_ms": {"p50": round(float(np.percentile(t["step_ms"], 50)), 3),
                             "p99": round(float(np.percentile(t["step_ms"], 99)), 3)},
              "recomputed_pairs": stats["recomputed_pairs"],
              "autotuned": tuned,
              "db_create_s": round(db_create_s, 3),
              "gpu_launches": stats["kernels_launched"] * args.steps,
              "clocks": clocks}

    sms = torch.cuda.get_device_properties(device).multi_processor_count
    rate, rate_mhz, _ = swgb.intpeak("viaddmax_s16x2", 8, 256, 20000)
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    peak = rate * sms * max_mhz * 1e6 / 1e12
    peak_src = (f"intpeak viaddmax_s16x2 {rate:.1f} lane-ops/clk/SM x {sms} SMs x "
                f"{max_mhz:.0f} MHz (max SM clock), measured")
    result["roofline"] = roofline(t, peak, peak_src, rate_mhz, lambda k: profiled_traffic(args, k))

    i32_rate, _, _ = swgb.intpeak("imax", 8, 256, 20000)
    result["paper_arch_efficiency"] = paper_arch_efficiency(gcups / world, i32_rate, sms, max_mhz)

    # plain int32 one-query-per-launch baseline on the same workload
    if not args.no_plain:
        pl, outp = plain_leg(d, q, w, device, stream)
        result["plain_int32"] = pl
        result["speedup_vs_plain"] = round(cells / (ms / 1e3) / 1e9 / pl["value"], 3)   # this rank
        result["plain_equals_packed"] = bool(torch.equal(outp, out))
        del outp

    # end to end through the C ABI with host buffers (pinned), copies timed
    e2e_s, out_host = e2e_leg(plan, q, N, w, min(args.steps, 3), dist, device)
    result["e2e"] = {"value": round(all_cells / e2e_s / 1e9, 2), "unit": "GCUPS",
                     "h2d_bytes_per_step": int(q.total + 4 * nq),
                     "d2h_bytes_per_step": int(4 * nq * N), "ms_per_step": round(1e3 * e2e_s, 3)}

    # one search split over the ranks (database sharded by cells, columns
    # all-gathered): strong scaling of the rank-0 workload
    if world > 1 and not args.no_shard:
        result["sharded"] = run_sharded(args, rank, world, local, device, dist,
                                        out if rank == 0 else None)

    # traceback of each query's best hit (sw_align), checked against the oracle
    if rank == 0 and world == 1 and args.workload in ("paper-search", "plain-small") and not args.no_align:
        result["align"] = run_align(d, q, db, out, w)

    # serving: the same resident DB, Poisson arrivals, continuous batching
    if args.serve > 0 and args.workload == "paper-search" and rank == 0 and world == 1:
        result["serving"] = run_serving(d, db, args, opts, w)

    # CPU oracle on a bounded sample (rank 0, N = 1): baseline and parity check
    if rank == 0 and world == 1 and not args.no_cpu:
        result["cpu_baseline"], result["parity_on_cpu_sample"] = cpu_leg(
            w, out_host.numpy(), args.cpu_cells or CPU_CELLS[args.workload])

    # the batched-uneven and long-sequence workloads, each measured in full
    # in the same run (one GPU, the default workload only)
    if (rank == 0 and world == 1 and args.workload == "paper-search" and not args.no_configs
            and not args.subjects and not args.queries):
        del out, out_host, plan
        d.close()
        torch.cuda.empty_cache()
        result["configs"] = {}
        for name in ("batched-uneven", "long"):
            result["configs"][name.replace("-", "_")] = run_config(
                name, args, device, local, stream, peak, peak_src, rate_mhz)
            torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
