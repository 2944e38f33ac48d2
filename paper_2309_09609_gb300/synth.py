"""Seeded synthetic protein workloads.

This module only draws inputs: residue codes, lengths and arrival times.  It
holds none of the alignment arithmetic, so both the CUDA path and the CPU
oracle may take their inputs from it.

The paper searches 20 Swiss-Prot queries (144-5478 residues) against the
Env-NR 2021_04 database (Section IV-A).  Neither is available here, so these
generators stand in for them with the same shapes:

* residues are i.i.d. over the 20 standard amino acids at the Robinson &
  Robinson (1991) background frequencies (the ones BLAST uses with BLOSUM62);
* database lengths are lognormal with mean 360 and median 290, rounded and
  clipped to [2, 35000];
* a small share of subjects is overwritten, at unchanged length, by mutated
  copies of query segments ("planted homologs"), so that high and saturating
  scores occur.

Codes follow the BLOSUM62 order A R N D C Q E G H I L K M F P S T W Y V B Z X *
(the 20 standard amino acids are codes 0..19).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

#: Robinson & Robinson (1991) amino-acid background frequencies, codes 0..19.
BACKGROUND = np.array([
    0.07805, 0.05129, 0.04487, 0.05364, 0.01925, 0.04264, 0.06295, 0.07377,
    0.02199, 0.05142, 0.09019, 0.05744, 0.02243, 0.03856, 0.05203, 0.07120,
    0.05841, 0.01330, 0.03216, 0.06441], dtype=np.float64)

#: lognormal subject lengths: median 290, mean 360
DB_MU = math.log(290.0)
DB_SIGMA = math.sqrt(2.0 * math.log(360.0 / 290.0))


def _residue_table() -> np.ndarray:
    # 65536-entry inverse-CDF table: residue = table[uniform uint16]
    cdf = np.cumsum(BACKGROUND / BACKGROUND.sum())
    u = (np.arange(65536, dtype=np.float64) + 0.5) / 65536.0
    return np.minimum(np.searchsorted(cdf, u, side="right"), 19).astype(np.uint8)


_TABLE = _residue_table()


def residues(rng: np.random.Generator, n: int, chunk: int = 1 << 24) -> np.ndarray:
    """n i.i.d. residue codes at background frequencies (uint8)."""
    out = np.empty(int(n), dtype=np.uint8)
    for lo in range(0, int(n), chunk):
        hi = min(int(n), lo + chunk)
        out[lo:hi] = _TABLE[rng.integers(0, 65536, size=hi - lo, dtype=np.uint16)]
    return out


def lognormal_lengths(rng, n, mu=DB_MU, sigma=DB_SIGMA, lo=2, hi=35000) -> np.ndarray:
    x = np.rint(rng.lognormal(mu, sigma, size=int(n)))
    return np.clip(x, lo, hi).astype(np.int32)


def uniform_lengths(rng, n, lo, hi) -> np.ndarray:
    return rng.integers(lo, hi + 1, size=int(n)).astype(np.int32)


def offsets(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(len(lengths), dtype=np.int64)
    if len(lengths) > 1:
        off[1:] = np.cumsum(lengths[:-1], dtype=np.int64)
    return off


@dataclass
class SeqSet:
    """Concatenated sequences: codes, per-sequence start offsets and lengths."""
    res: np.ndarray      # uint8 [sum(lens)]
    lens: np.ndarray     # int32 [n]
    offs: np.ndarray = field(default=None)  # int64 [n]

    def __post_init__(self):
        self.res = np.ascontiguousarray(self.res, dtype=np.uint8)
        self.lens = np.ascontiguousarray(self.lens, dtype=np.int32)
        if self.offs is None:
            self.offs = offsets(self.lens)

    def __len__(self):
        return int(self.lens.size)

    def seq(self, i: int) -> np.ndarray:
        o = int(self.offs[i])
        return self.res[o:o + int(self.lens[i])]

    @property
    def total(self) -> int:
        return int(self.lens.sum(dtype=np.int64))

    def subset(self, idx) -> "SeqSet":
        idx = np.asarray(idx, dtype=np.int64)
        lens = self.lens[idx]
        parts = [self.seq(int(i)) for i in idx]
        res = np.concatenate(parts) if parts and lens.sum() else np.zeros(0, np.uint8)
        return SeqSet(res, lens)


def random_seqset(rng, lens) -> SeqSet:
    lens = np.asarray(lens, dtype=np.int32)
    return SeqSet(residues(rng, int(lens.sum(dtype=np.int64))), lens)


def mutate(rng, seq: np.ndarray, rate: float) -> np.ndarray:
    """Point mutations: each position redrawn at background with prob. rate."""
    out = seq.copy()
    hit = rng.random(seq.size) < rate
    out[hit] = residues(rng, int(hit.sum()))
    return out


def plant_homologs(rng, db: SeqSet, sources: SeqSet, count: int,
                   rate_lo=0.10, rate_hi=0.20, prefer_long=False) -> np.ndarray:
    """Overwrite `count` subjects in place with mutated source segments.

    Lengths do not change: a subject no longer than the source receives a
    random window of the mutated source; a longer subject receives the whole
    mutated source at a random offset.  Returns the planted subject indices.
    """
    n = len(db)
    if count <= 0 or n == 0 or len(sources) == 0:
        return np.zeros(0, dtype=np.int64)
    if prefer_long:
        cand = np.argsort(db.lens, kind="stable")[::-1][:max(count * 4, count)]
        idx = rng.choice(cand, size=min(count, cand.size), replace=False)
    else:
        idx = rng.choice(n, size=min(count, n), replace=False)
    src_order = np.argsort(sources.lens, kind="stable")[::-1]
    for k, s in enumerate(np.sort(idx)):
        src = sources.seq(int(src_order[k % len(sources)] if prefer_long
                              else rng.integers(len(sources))))
        mut = mutate(rng, src, float(rng.uniform(rate_lo, rate_hi)))
        o, L = int(db.offs[s]), int(db.lens[s])
        if L <= mut.size:
            a = int(rng.integers(0, mut.size - L + 1))
            db.res[o:o + L] = mut[a:a + L]
        else:
            a = int(rng.integers(0, L - mut.size + 1))
            db.res[o + a:o + a + mut.size] = mut
    return np.sort(idx).astype(np.int64)


@dataclass
class Workload:
    name: str
    queries: SeqSet
    db: SeqSet
    gap_open: int = 10
    gap_extend: int = 2
    planted: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    note: str = ""

    @property
    def cells(self) -> int:
        return self.queries.total * self.db.total


# ---- the five workload shapes ------------------------------------------------

def plain_small(seed: int = 0) -> Workload:
    """One 144-residue query vs 2,000 subjects of length U[50, 1000]."""
    rng = np.random.default_rng(seed)
    q = random_seqset(rng, [144])
    db = random_seqset(rng, uniform_lengths(rng, 2000, 50, 1000))
    return Workload("plain-small: 1 query (144) x 2,000 subjects U[50,1000]", q, db)


def paper_query_lengths(n: int = 20, lo: int = 144, hi: int = 5478) -> np.ndarray:
    """Log-spaced query lengths lo..hi (the paper's 20 queries span 144-5478)."""
    k = np.arange(n, dtype=np.float64)
    return np.rint(lo * (hi / lo) ** (k / max(n - 1, 1))).astype(np.int32)


def paper_search(seed: int = 0, n_subjects: int = 570_000, n_queries: int = 20,
                 plant_frac: float = 1e-4) -> Workload:
    """20 log-spaced queries (144-5478) vs a lognormal DB (mean 360)."""
    rng = np.random.default_rng(seed)
    q = random_seqset(rng, paper_query_lengths(n_queries))
    db = random_seqset(rng, lognormal_lengths(rng, n_subjects))
    planted = plant_homologs(rng, db, q, max(1, int(round(plant_frac * n_subjects))))
    return Workload(f"paper-search: {n_queries} queries (144-5478, log-spaced) x "
                    f"{n_subjects:,} lognormal subjects (mean 360)", q, db,
                    planted=planted, note=f"{planted.size} planted homologs")


def batched_uneven(seed: int = 0, n_queries: int = 1000, n_subjects: int = 100_000) -> Workload:
    """1,000 queries U[50, 2000] vs a 100,000-subject lognormal DB."""
    rng = np.random.default_rng(seed)
    q = random_seqset(rng, uniform_lengths(rng, n_queries, 50, 2000))
    db = random_seqset(rng, lognormal_lengths(rng, n_subjects))
    planted = plant_homologs(rng, db, q, max(1, int(round(1e-4 * n_subjects))))
    return Workload(f"batched-uneven: {n_queries} queries U[50,2000] x {n_subjects:,} "
                    "lognormal subjects", q, db, planted=planted)


def long_sequences(seed: int = 0, n_queries: int = 8, n_subjects: int = 20_000,
                   lo: int = 5000, hi: int = 35000, n_planted: int = 4) -> Workload:
    """8 queries and 20,000 subjects, all of length U[5000, 35000]."""
    rng = np.random.default_rng(seed)
    q = random_seqset(rng, uniform_lengths(rng, n_queries, lo, hi))
    db = random_seqset(rng, uniform_lengths(rng, n_subjects, lo, hi))
    planted = plant_homologs(rng, db, q, n_planted, 0.05, 0.10, prefer_long=True)
    return Workload(f"long: {n_queries} queries x {n_subjects:,} subjects, U[{lo},{hi}]",
                    q, db, planted=planted, note=f"{planted.size} planted homologs")


@dataclass
class Arrivals:
    times: np.ndarray      # seconds from the start, non-decreasing
    queries: SeqSet


def serving_trace(seed: int = 0, n: int = 1000, rate: float = 50.0,
                  mean_len: float = 400.0, lo: int = 30, hi: int = 5000) -> Arrivals:
    """Poisson arrivals at `rate`/s; query lengths lognormal (mean 400)."""
    rng = np.random.default_rng(seed + 7919)
    times = np.cumsum(rng.exponential(1.0 / rate, size=int(n)))
    sigma = DB_SIGMA
    mu = math.log(mean_len) - sigma * sigma / 2.0
    lens = lognormal_lengths(rng, n, mu, sigma, lo, hi)
    return Arrivals(times, random_seqset(rng, lens))
