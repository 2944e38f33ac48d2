"""bench.py under two ranks, end to end with the CUDA library: each rank's
own seeded search (weak scaling), the split search of the one-GPU workload
with its gathered columns checked against rank 0's one-GPU scores, and one
JSON line from rank 0.  This run has one GPU, so both ranks use it (their
searches are independent; the collectives are gloo's, on the host): the
timings mean nothing here, the code path is what is tested."""
import json
import os
import socket
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_ranks_print_one_line_with_the_split_search_checked():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK="0", WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), SWGB_BENCH_BACKEND="gloo")
        procs.append(subprocess.Popen(
            [sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--workload",
             "plain-small", "--steps", "2", "--warmup", "1", "--no-configs", "--serve", "0",
             "--no-cpu", "--no-align"],
            env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=600) for p in procs]
    for p, (out, err) in zip(procs, outs):
        assert p.returncode == 0, err[-3000:]
    line = json.loads([l for l in outs[0][0].splitlines() if l.startswith("{")][-1])
    # rank 1 prints no result line (a library may log a connection line)
    assert not [l for l in outs[1][0].splitlines() if l.startswith("{")]
    assert line["n_gpus"] == 2 and line["scaling"] == "weak" and line["value"] > 0
    sh = line["sharded"]
    assert sh["equals_one_gpu"] is True and sh["scaling"] == "strong"
    assert sum(sh["subjects_per_rank"]) == line["config"]["subjects"]
    assert min(sh["residues_per_rank"]) > 0
