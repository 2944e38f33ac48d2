"""One search split over two ranks with the CUDA library on each (Section
III-A multi-GPU policy): each rank searches its cell-weighted partition of
the database on the GPU, the int32 columns are all-gathered (gloo, on the
host), and every rank ends with the oracle's full score matrix.

This run has one GPU, so both ranks use it; their searches are independent
(no kernel of one rank waits on the other's), and only the host-side gather
joins them."""
import os
import socket
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
    from helpers import oracle_all
    from paper_2309_09609_gb300 import shard, swgb, synth
    dist.init_process_group("gloo")
    rank = dist.get_rank()
    rng = np.random.default_rng(5)                       # the same inputs on both ranks
    db = synth.random_seqset(rng, np.concatenate([synth.lognormal_lengths(rng, 6000),
                                                  [0, 1, 2600, 4000]]))
    q = synth.random_seqset(rng, [37, 144, 300, 555, 1000])
    want = oracle_all(q, db, 10, 2) if rank == 0 else None
    for weights in ([1, 1], [1, 2]):
        sd = shard.ShardedDatabase(db, dist, weights=weights, device=0)
        assert isinstance(sd.db, swgb.Database)
        got = sd.search(q.res, q.lens, 10, 2)
        if rank == 0:
            assert got.shape == want.shape and (got == want).all(), weights
        got2 = sd.search(q.res, q.lens, 11, 1)            # the plan is reused
        if rank == 0:
            assert (got2 == oracle_all(q, db, 11, 1)).all()
    dist.barrier()
    dist.destroy_process_group()
    print("ok", rank)
""")


def test_two_ranks_on_the_gpu_gather_the_oracle_matrix():
    pytest.importorskip("torch")
    from paper_2309_09609_gb300 import build as nvbuild
    nvbuild.build()
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK="0", WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=600)[0] for p in procs]
    for rank, (p, out) in enumerate(zip(procs, outs)):
        assert p.returncode == 0, out
        assert f"ok {rank}" in out
