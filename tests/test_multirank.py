"""The N > 1 host path of bench.py on CPU: two gloo ranks, barrier, the
max-over-ranks timing reduction and the sum of the cells the ranks scored
(each rank runs its own seeded search of the same shape; the search itself
has no collective)."""
import os
import socket
import subprocess
import sys
import textwrap

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
    os.environ["SWGB_BENCH_BACKEND"] = "gloo"
    import bench
    rank, world, local, dist = bench.dist_setup(None)
    assert world == 2 and dist is not None
    dist.barrier()
    t = bench.max_over_ranks(10.0 + rank, dist, "cpu")
    assert t == 11.0, t
    c = bench.sum_over_ranks(1e12 * (1 + rank), dist, "cpu")
    assert c == 3e12, c
    # each rank its own search of the same shape; rank 0 = the one-GPU workload
    import argparse
    a = argparse.Namespace(workload="plain-small", seed=0, subjects=None, queries=None,
                           query_offset=0)
    w = bench.rank_workload(a, rank)
    w0 = bench.make_workload("plain-small", 0)
    assert len(w.db) == len(w0.db) and len(w.queries) == len(w0.queries)
    assert (w.db.res.size == w0.db.res.size and (w.db.res == w0.db.res).all()) == (rank == 0)
    dist.barrier()
    dist.destroy_process_group()
    print("ok", rank)
""")


def test_two_gloo_ranks_reduce_time_and_cells():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                                      text=True))
    outs = [p.communicate(timeout=120)[0] for p in procs]
    for rank, (p, out) in enumerate(zip(procs, outs)):
        assert p.returncode == 0, out
        assert f"ok {rank}" in out


def test_reference_arm_runs_on_rank_zero_only():
    # bench.py --impl reference under two ranks: rank 0 times the oracle and
    # prints the one JSON line; rank 1 exits 0 without work or output
    import json
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), SWGB_BENCH_BACKEND="gloo")
        procs.append(subprocess.Popen(
            [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
             "--workload", "plain-small", "--steps", "1", "--warmup", "0", "--ref-cells", "2e7"],
            env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    for p, (out, err) in zip(procs, outs):
        assert p.returncode == 0, err
    line = json.loads(outs[0][0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    # the same workload keys as the GPU arm's config
    import bench
    w = bench.make_workload("plain-small", 0)
    cfg = line["config"]
    assert {k: cfg[k] for k in bench.workload_config(w)} == bench.workload_config(w)
    assert outs[1][0].strip() == ""
