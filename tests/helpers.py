"""Test helpers: oracle scores for SeqSet inputs, random inputs."""
import numpy as np

import oracle
from paper_2309_09609_gb300 import synth


def oracle_all(q, db, gap_open=10, gap_extend=2, matrix=None, nthreads=None):
    nq, nd = len(q), len(db)
    pq = np.repeat(np.arange(nq, dtype=np.int32), nd)
    pd = np.tile(np.arange(nd, dtype=np.int64), nq)
    return oracle.pairs_packed(q.res, q.offs, q.lens, db.res, db.offs, db.lens, pq, pd,
                               gap_open, gap_extend, matrix, nthreads).reshape(nq, nd)


def oracle_pairs(q, db, pq, pd, gap_open=10, gap_extend=2, matrix=None):
    return oracle.pairs_packed(q.res, q.offs, q.lens, db.res, db.offs, db.lens,
                               np.asarray(pq, np.int32), np.asarray(pd, np.int64),
                               gap_open, gap_extend, matrix)


def seqset(rng, lens, alpha=20):
    lens = np.asarray(lens, dtype=np.int32)
    if alpha == 20:
        return synth.random_seqset(rng, lens)
    res = rng.integers(0, alpha, size=int(lens.sum())).astype(np.uint8)
    return synth.SeqSet(res, lens)


def rand_matrix(rng, lo=-5, hi=9, symmetric=False):
    a = rng.integers(lo, hi + 1, size=(24, 24))
    if symmetric:
        a = np.triu(a) + np.triu(a, 1).T
    return a.astype(np.int8)


def from_text(*seqs):
    arrs = [oracle.encode(s) for s in seqs]
    return synth.SeqSet(np.concatenate(arrs) if arrs else np.zeros(0, np.uint8),
                        np.array([a.size for a in arrs], np.int32))


def concat(*sets):
    res = np.concatenate([s.res for s in sets])
    lens = np.concatenate([s.lens for s in sets])
    return synth.SeqSet(res, lens)
