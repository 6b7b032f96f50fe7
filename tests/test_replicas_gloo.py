"""The multi-GPU bench path is replicas only (one independent problem per rank,
no data-path collective): its host logic, run as two gloo ranks on the CPU —
the max over ranks that the job's time is, the per-rank seeding of the replicas,
and the reference arm, which only rank 0 runs."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"])
dist.init_process_group("gloo", rank=rank, world_size=2)
mx = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
class A: workload = "rbf_small"; n = 300
wl = bench.workload(A, seed=rank)
print(json.dumps({"rank": rank, "max": mx, "x00": float(wl.X[0, 0]),
                  "value": bench.job_throughput_value(mx * 1e3, 2, 3)}), flush=True)
dist.barrier()
dist.destroy_process_group()
"""


def test_two_gloo_ranks_take_the_max_and_seed_replicas_apart():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(__import__("json").loads(out.strip().splitlines()[-1]))
    assert all(o["max"] == 15.0 for o in outs)
    assert outs[0]["x00"] != outs[1]["x00"]               # replicas are independent problems
    assert outs[0]["value"] == pytest.approx(15.0 / 6)    # seconds per solve over 2 ranks x 3 steps


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
