"""Multi-rank (replica) host logic on CPU: two gloo ranks join the group from the launcher's
environment, take the max of per-rank timings, meet at barriers and get disjoint instance
seeds -- the N > 1 path of bench.py without a GPU.  Also runs bench.py's reference arm
under two ranks: rank 0 prints one line, rank 1 exits cleanly without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import json, os, sys
sys.path.insert(0, %(root)r)
from paper_1911_03225_gb300 import replicas
world, rank, local = replicas.init_replicas("gloo")
t = replicas.max_over_ranks(1.5 + rank, world)
replicas.barrier(world)
seeds = replicas.instance_seeds(4, rank)
import torch, torch.distributed as dist
g = [None] * world
dist.all_gather_object(g, seeds)
with open(os.path.join(%(out)r, "rank%%d.json" %% rank), "w") as f:
    json.dump({"rank": rank, "world": world, "local": local, "max": t, "seeds": seeds, "all": g}, f)
replicas.finalize(world)
"""


def launch(code_or_args, nproc=2, timeout=180):
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", str(nproc),
           "--master-addr", "127.0.0.1", "--master-port", str(port)] + code_or_args
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def test_two_gloo_ranks_max_barrier_and_disjoint_seeds(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(WORKER % {"root": ROOT, "out": str(tmp_path)})
    r = launch([str(script)])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.load(open(tmp_path / ("rank%d.json" % k))) for k in range(2)]
    assert sorted(d["rank"] for d in lines) == [0, 1]
    for d in lines:
        assert d["world"] == 2 and d["max"] == 2.5
        assert d["all"] == [[0, 1, 2, 3], [4, 5, 6, 7]]


def test_reference_arm_under_two_ranks_prints_one_line():
    r = launch(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"], timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["unit"] == "cell-steps/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
