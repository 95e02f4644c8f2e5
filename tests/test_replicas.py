"""The N > 1 path of the benchmark on the host: one process per rank (gloo on CPU,
world size 2), the slowest rank's time shared by every rank, the whole-job throughput
summed over the replicas, and the reference arm running on rank 0 only."""
import argparse
import json
import os
import socket
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank = dist.get_rank()
ms_local = 10.0 + 7.5 * rank              # rank 1 is the slow one
ms = bench.max_over_ranks(ms_local, dist, "cpu")
dist.barrier()
value = bench.job_throughput(20, 3, dist.get_world_size(), ms)
print(json.dumps({"rank": rank, "ms": ms, "value": value}))
dist.destroy_process_group()
"""


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_max_over_ranks_and_job_throughput_gloo_world2():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), REPO_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", _RANK_SCRIPT], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["ms"] == 17.5  # the slowest rank's time on every rank
        # 2 replicas x 3 solves x 20 pairs in 17.5 ms
        assert abs(o["value"] - 2 * 3 * 20 / 0.0175) < 1e-9 * o["value"]


def test_single_rank_time_is_its_own():
    assert bench.max_over_ranks(12.25, None, "cpu") == 12.25
    assert bench.job_throughput(20, 30, 1, 204.0) == 20 * 30 / 0.204


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(impl="reference", gpus=2, steps=1, warmup=0)
    assert bench.run_reference(args) == 0  # rank 1 returns before any work
    assert capsys.readouterr().out == ""
