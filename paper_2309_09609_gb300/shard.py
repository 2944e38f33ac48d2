"""One search over several GPUs: the database split by cells, the score
columns gathered back in caller order.

The paper runs its multi-GPU searches by splitting the work between the GPUs
and observes that an unweighted split leaves the faster GPU idle (Section
III-A's multi-GPU policy; Section IV-C and Table IV: two different GPUs reach
less than the sum of their single-GPU rates).  Here the database is split
into contiguous partitions of the caller's subject order, one per rank, each
holding a share of the residues proportional to the rank's weight (equal
for identical GPUs, or each GPU's measured GCUPS).  A search's cells on a
rank are the batch's query residues times the partition's residues, so the
shares of cells follow the weights, within one subject per boundary.

Each rank searches its partition with the unchanged one-GPU library (a
database and a plan of its own); there is no exchange until the end, where
the int32 score columns of every rank are all-gathered (NCCL between GPUs,
gloo on the CPU), padded to the longest partition and trimmed, so that every
rank ends with the full score matrix in caller order.
"""
from __future__ import annotations

import numpy as np


def partition(lengths, weights) -> np.ndarray:
    """Boundaries b[0] = 0 <= b[1] <= ... <= b[R] = N of R contiguous
    partitions of the subjects: partition r holds subjects [b[r], b[r+1]),
    whose residues come as close as a subject boundary allows to the share
    weights[r] / sum(weights) of all residues (each boundary is the prefix
    whose residue count is nearest its target, so a partition's residues
    differ from its share by at most the longest subject)."""
    lengths = np.asarray(lengths, dtype=np.int64)
    w = np.asarray(weights, dtype=np.float64)
    if w.ndim != 1 or w.size < 1 or not np.all(np.isfinite(w)) or np.any(w <= 0):
        raise ValueError("weights must be positive, one per rank")
    prefix = np.zeros(lengths.size + 1, dtype=np.int64)
    np.cumsum(lengths, out=prefix[1:])
    total = int(prefix[-1])
    targets = total * np.cumsum(w)[:-1] / w.sum()
    bounds = [0]
    for t in targets:
        i = int(np.searchsorted(prefix, t, side="left"))   # prefix[i] >= t
        i = min(i, lengths.size)
        if i > 0 and t - prefix[i - 1] <= prefix[i] - t:   # the nearer prefix
            i -= 1
        bounds.append(max(i, bounds[-1]))
    bounds.append(lengths.size)
    return np.array(bounds, dtype=np.int64)


class ShardedDatabase:
    """This rank's partition of a database, and the search that gathers
    every rank's columns.

    ``subjects`` is a ``synth.SeqSet``-like object (``res``, ``lens``,
    ``offs``, ``subset``) holding the whole database in caller order, the
    same on every rank.  ``dist`` is ``torch.distributed`` with its process
    group initialised (or None for one rank).  ``make_db(seqset, device)``
    builds the rank's database (default: the CUDA library's)."""

    def __init__(self, subjects, dist=None, weights=None, device: int = 0, make_db=None,
                 **plan_opts):
        self.dist = dist
        self.rank = dist.get_rank() if dist is not None else 0
        self.world = dist.get_world_size() if dist is not None else 1
        self.n = len(subjects)
        self.weights = np.ones(self.world) if weights is None else np.asarray(weights, float)
        if self.weights.size != self.world:
            raise ValueError("one weight per rank")
        self.bounds = partition(subjects.lens, self.weights)
        lo, hi = int(self.bounds[self.rank]), int(self.bounds[self.rank + 1])
        self.local = subjects.subset(np.arange(lo, hi))
        self.device = device
        if make_db is None:
            from . import swgb
            make_db = lambda ss, dev: swgb.Database.from_seqset(ss, device=dev)  # noqa: E731
        self.db = make_db(self.local, device)
        self.plan_opts = plan_opts
        self._plan = None

    @property
    def sizes(self) -> np.ndarray:
        return np.diff(self.bounds)

    def _local_scores(self, queries, q_lengths, gap_open, gap_extend, matrix):
        q = np.ascontiguousarray(queries, dtype=np.uint8)
        ql = np.ascontiguousarray(q_lengths, dtype=np.int32)
        if not hasattr(self.db, "plan"):          # a stand-in database (tests)
            return self.db.search(q, ql, gap_open, gap_extend, matrix)
        cap = (max(ql.size, 1), max(int(ql.sum()), 1))
        if self._plan is None or self._plan.max_queries < cap[0] or \
                self._plan.max_query_residues < cap[1]:
            self._plan = self.db.plan(*cap, **self.plan_opts)
        return self._plan.search(q, ql, gap_open, gap_extend, matrix)

    def search(self, queries, q_lengths, gap_open=10, gap_extend=2, matrix=None) -> np.ndarray:
        """Every query against every subject of the whole database: int32
        [n_queries, n_subjects] in caller order, on the host, on every rank."""
        local = np.asarray(self._local_scores(queries, q_lengths, gap_open, gap_extend, matrix),
                          dtype=np.int32)
        nq = int(np.asarray(q_lengths).size)
        if self.dist is None or self.world == 1:
            return local.reshape(nq, self.n)
        return self.gather(local.reshape(nq, -1))

    def gather(self, local: np.ndarray) -> np.ndarray:
        """All-gathers every rank's [nq, n_r] columns into [nq, N], caller order."""
        import torch
        nq = local.shape[0]
        width = int(self.sizes.max()) if self.sizes.size else 0
        backend = self.dist.get_backend()
        dev = torch.device("cuda", self.device) if backend == "nccl" else torch.device("cpu")
        buf = torch.zeros((nq, width), dtype=torch.int32, device=dev)
        buf[:, :local.shape[1]] = torch.from_numpy(local).to(dev)
        parts = [torch.empty_like(buf) for _ in range(self.world)]
        self.dist.all_gather(parts, buf)
        cols = [p[:, :int(s)] for p, s in zip(parts, self.sizes)]
        return torch.cat(cols, dim=1).cpu().numpy() if cols else np.zeros((nq, 0), np.int32)
