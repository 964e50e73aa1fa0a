"""The bench's multi-rank plumbing on CPU: world size 2 over gloo, 127.0.0.1.

Each rank of `bench.py --gpus N` runs its own jet (weak scaling, no data-path
collective); the whole-job time is the maximum over ranks, and only rank 0
prints.  These checks run the same helpers with two CPU processes.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
ws, rank, local = bench.dist_env()
t = bench.max_over_ranks(1.0 + rank, ws)        # rank 1 is the slow one
bench.barrier(ws)
seeds = [None] * ws
dist.all_gather_object(seeds, bench.workload(seed=1234 + rank)["params"]["seed"])
print(json.dumps({{"rank": rank, "ws": ws, "max": t, "seeds": seeds}}))
dist.destroy_process_group()
"""


def _launch(code, n=2, extra_env=None):
    port = _free_port()
    procs = []
    for r in range(n):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(n), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), **(extra_env or {}))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=240)
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_max_over_ranks_and_independent_jets():
    outs = _launch(WORKER.format(root=ROOT))
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for r in res:
        assert r["ws"] == 2
        assert r["max"] == 2.0            # the slowest rank sets the whole-job time
        assert r["seeds"] == [1234, 1235]  # each rank runs its own jet


def test_reference_arm_prints_on_rank_zero_only():
    code = f"import sys; sys.path.insert(0, {ROOT!r}); sys.argv = ['bench.py', '--impl', 'reference', '--steps', '1', " \
           f"'--warmup', '3']; import bench; sys.exit(bench.main())"
    outs = _launch(code)
    line = json.loads(outs[0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["cpu_baseline"]["kind"] == "oracle"
    assert outs[1].strip() == ""
