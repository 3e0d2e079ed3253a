"""Host-side partition of a batch of independent images over ranks (wmc_shard_lpt): the
longest-processing-time-first rule, pinned by a hand example, Graham's bound against a
brute-force optimum on small instances, and two gloo ranks that compute the same partition
independently.  No GPU: the function makes no CUDA call."""
import itertools
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from paper_1903_07189_gb300 import synth, wmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_hand_example_shows_the_greedy_order():
    # decreasing costs 5, 4, 3, 3, 3 on two ranks: 5 -> r0, 4 -> r1, 3 -> r1 (4 < 5),
    # 3 -> r0 (5 < 7), 3 -> r1 (7 < 8); loads 8 and 10, where {5, 4} / {3, 3, 3} would give 9 / 9
    owner, load = wmc.shard_lpt([5, 4, 3, 3, 3], 2)
    assert owner == [0, 1, 1, 0, 1]
    assert load == [8, 10]


def test_equal_costs_go_round_robin_in_index_order():
    owner, load = wmc.shard_lpt([2, 2, 2, 2], 3)
    assert owner == [0, 1, 2, 0]
    assert load == [4, 2, 2]
    # the sort is by cost only: an image's position among equal costs is its index
    owner, _ = wmc.shard_lpt([1, 7, 1, 7], 2)
    assert owner == [0, 0, 1, 1]


def test_degenerate_arguments():
    assert wmc.shard_lpt([], 4) == ([], [0, 0, 0, 0])
    owner, load = wmc.shard_lpt([3, 1, 4, 1, 5], 1)
    assert owner == [0] * 5 and load == [14]
    owner, load = wmc.shard_lpt([9, 8], 5)  # more ranks than images: the rest stay empty
    assert owner == [0, 1] and load == [9, 8, 0, 0, 0]
    for bad in ([[1, 2], 0], [[1, -1], 2]):
        with pytest.raises(RuntimeError):
            wmc.shard_lpt(*bad)


def brute_force_best(costs, world):
    best = None
    for assign in itertools.product(range(world), repeat=len(costs)):
        loads = [0] * world
        for c, r in zip(costs, assign):
            loads[r] += c
        m = max(loads)
        best = m if best is None else min(best, m)
    return best


@pytest.mark.parametrize("world", [2, 3])
def test_grahams_bound_against_the_optimum(world):
    rng = np.random.default_rng(11)
    for _ in range(40):
        n = int(rng.integers(1, 9))
        costs = [int(x) for x in rng.integers(1, 100, n)]
        owner, load = wmc.shard_lpt(costs, world)
        assert sorted(set(owner)) <= list(range(world))
        assert load == [sum(c for c, r in zip(costs, owner) if r == k) for k in range(world)]
        opt = brute_force_best(costs, world)
        assert max(load) * 3 * world <= opt * (4 * world - 1), (costs, load, opt)


def test_batch_workload_partition():
    """The 512 images of the batch workload (sides 64..1536) by pixel count: every image on one
    rank, and the largest load within 1 % of the mean for 2 to 8 ranks."""
    sizes = synth.batch_sizes(512)
    costs = [h * w for h, w in sizes]
    for world in (2, 4, 8):
        owner, load = wmc.shard_lpt(costs, world)
        assert sum(load) == sum(costs)
        assert max(load) <= 1.01 * sum(costs) / world


WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["WMC_ROOT"])
import torch.distributed as dist
from paper_1903_07189_gb300 import synth, wmc
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
costs = [h * w for h, w in synth.batch_sizes(512)]
owner, _ = wmc.shard_lpt(costs, world)
mine = [i for i, r in enumerate(owner) if r == rank]
got = [None] * world
dist.all_gather_object(got, {"owner": owner, "mine": mine})
dist.barrier()
dist.destroy_process_group()
print(json.dumps(got))
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_compute_the_same_partition():
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), WMC_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert outs[0] == outs[1]
    views = outs[0]
    assert views[0]["owner"] == views[1]["owner"]
    mine = sorted(views[0]["mine"] + views[1]["mine"])
    assert mine == list(range(512))  # every image on exactly one rank
