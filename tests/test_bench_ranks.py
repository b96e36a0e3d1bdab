"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the job time is the slowest
rank's, the job rate counts every rank's units, and the reference arm runs on rank 0 only.
The path shards by atmosphere with no exchange, so these are the only cross-rank steps."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
local_ms = [3.0, 5.0][rank]
t = bench.max_over_ranks(dist, local_ms)
rate = bench.job_rate(world, 100, t)
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "t_max": t, "rate": rate}))
"""


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_max_over_ranks_and_job_rate_gloo():
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), REPO_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["t_max"] == 5.0                       # the slower rank's time
        assert o["rate"] == 2 * 100 / 5e-3             # both ranks' units over that time


def test_single_process_helpers():
    import bench
    assert bench.max_over_ranks(None, 7.5) == 7.5
    assert bench.job_rate(1, 1000, 250.0) == 4000.0


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
