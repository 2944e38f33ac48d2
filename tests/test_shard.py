"""Database sharding across ranks (paper Section III-A multi-GPU policy,
Section IV-C): the cell-weighted partition, and one search split over two
gloo ranks whose gathered score matrix equals the oracle's.  On the CPU each
rank scores its partition with the oracle in place of the GPU library."""
import os
import socket
import subprocess
import sys
import textwrap

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2309_09609_gb300 import shard, synth  # noqa: E402


@pytest.mark.parametrize("weights", [[1, 1], [1, 3], [2, 1, 1], [1] * 8, [5, 1, 1, 1, 2]])
def test_partition_covers_every_subject_once_within_one_subject_of_its_share(weights):
    rng = np.random.default_rng(len(weights))
    lens = synth.lognormal_lengths(rng, 10000)
    b = shard.partition(lens, weights)
    assert b[0] == 0 and b[-1] == lens.size and np.all(np.diff(b) >= 0)
    assert b.size == len(weights) + 1
    res = np.array([lens[b[r]:b[r + 1]].sum() for r in range(len(weights))], dtype=np.int64)
    assert res.sum() == lens.sum()                      # every subject exactly once
    share = lens.sum() * np.asarray(weights, float) / np.sum(weights)
    assert np.all(np.abs(res - share) <= lens.max())   # cells follow the weights


def test_partition_edges():
    assert shard.partition([], [1, 1]).tolist() == [0, 0, 0]
    assert shard.partition([5], [1, 1, 1]).tolist()[-1] == 1
    b = shard.partition([0, 0, 7, 0, 3], [1, 1])
    assert b[0] == 0 and b[-1] == 5
    assert shard.partition([4, 4, 4, 4], [1, 1, 1, 1]).tolist() == [0, 1, 2, 3, 4]
    assert shard.partition([4, 4, 4, 4], [3, 1]).tolist() == [0, 3, 4]
    for bad in ([], [1, 0], [1, -1], [np.nan]):
        with pytest.raises(ValueError):
            shard.partition([1, 2, 3], bad)


def test_one_rank_needs_no_collective():
    import oracle
    rng = np.random.default_rng(3)
    db = synth.random_seqset(rng, rng.integers(1, 300, 50))
    q = synth.random_seqset(rng, [20, 70])

    class OracleDb:
        def __init__(self, ss, device):
            self.ss = ss

        def search(self, qres, qlen, go, ge, matrix):
            qs = synth.SeqSet(qres, qlen)
            return oracle.search([qs.seq(i) for i in range(len(qs))],
                                 [self.ss.seq(j) for j in range(len(self.ss))], go, ge, matrix)

    sd = shard.ShardedDatabase(db, None, make_db=OracleDb)
    got = sd.search(q.res, q.lens)
    want = oracle.search([q.seq(i) for i in range(2)], [db.seq(j) for j in range(50)])
    assert (got == want).all() and sd.sizes.tolist() == [50]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


CHILD = textwrap.dedent("""
    import os, sys
    sys.path.insert(0, {root!r})
    sys.path.insert(0, os.path.join({root!r}, "tests"))
    import numpy as np
    import torch.distributed as dist
    import oracle
    from helpers import oracle_all
    from paper_2309_09609_gb300 import shard, synth
    dist.init_process_group("gloo")
    rank = dist.get_rank()

    class OracleDb:
        # stands in for the rank's GPU database: the oracle on its partition
        def __init__(self, ss, device):
            self.ss = ss

        def search(self, qres, qlen, go, ge, matrix):
            return oracle_all(synth.SeqSet(qres, qlen), self.ss, go, ge, matrix)

    rng = np.random.default_rng(11)                       # the same inputs on both ranks
    db = synth.random_seqset(rng, np.concatenate([rng.integers(0, 400, 300), [0, 1, 2500]]))
    q = synth.random_seqset(rng, [1, 33, 144, 400])
    want = oracle_all(q, db, 10, 2)
    for weights in ([1, 1], [1, 3]):
        sd = shard.ShardedDatabase(db, dist, weights=weights, make_db=OracleDb)
        got = sd.search(q.res, q.lens, 10, 2)
        assert got.shape == want.shape and (got == want).all(), weights
        res = [int(db.lens[sd.bounds[r]:sd.bounds[r + 1]].sum()) for r in range(2)]
        share = db.total * np.array(weights) / sum(weights)
        assert all(abs(a - b) <= db.lens.max() for a, b in zip(res, share)), (res, share)
    # another scoring, through the same partitions
    m = rng.integers(-4, 8, size=(24, 24)).astype(np.int32)
    sd = shard.ShardedDatabase(db, dist, make_db=OracleDb)
    assert (sd.search(q.res, q.lens, 5, 1, m) == oracle_all(q, db, 5, 1, m)).all()
    dist.barrier()
    dist.destroy_process_group()
    print("ok", rank)
""")


def test_two_gloo_ranks_gather_the_full_matrix():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=300)[0] for p in procs]
    for rank, (p, out) in enumerate(zip(procs, outs)):
        assert p.returncode == 0, out
        assert f"ok {rank}" in out
