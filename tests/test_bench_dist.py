"""The benchmark's multi-rank logic on the host: two gloo ranks (world size 2, CPU) agree on
the slowest rank's time, compute the whole-job rate from it, get different replica inputs, and
the reference arm does its work on rank 0 only.  Replicas share no data, so this is all the
multi-rank path there is."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["WMC_ROOT"])
import torch, torch.distributed as dist
import bench
rank, world, _ = bench.dist_env()
dist.init_process_group("gloo", rank=rank, world_size=world)
local_ms = 10.0 + 5.0 * rank
slowest = bench.max_over_ranks(local_ms, world, torch.device("cpu"))
rate = bench.job_rate(1e9, world, slowest)
dist.barrier()
print(json.dumps({"rank": rank, "slowest": slowest, "rate": rate, "seed": bench.replica_seed(rank)}))
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_agree_on_slowest_time_and_rate():
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WMC_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert [o["slowest"] for o in outs] == [15.0, 15.0]
    # 2 ranks x 1e9 units in 15 ms
    assert all(abs(o["rate"] - 2e9 / 15e-3 / 1e9) < 1e-9 for o in outs)
    assert outs[0]["seed"] != outs[1]["seed"]


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.job_rate(2e9, 1, 1000.0) == pytest.approx(2.0)


def test_replicas_get_distinct_inputs():
    from paper_1903_07189_gb300 import synth
    a = synth.make_image(64, 64, seed=bench.replica_seed(0))
    b = synth.make_image(64, 64, seed=bench.replica_seed(1))
    assert not np.array_equal(a, b)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1"])
    assert bench.main() == 0
    assert capsys.readouterr().out == ""
