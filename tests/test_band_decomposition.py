"""Row-band decomposition of the Jacobi flow (Sec. V-B), checked on the CPU with gloo ranks.

A rank owns a band of image rows and keeps T extra rows on each side that it does not own.
Every round it takes the neighbours' rows of U^{rT} into those halos (one send/receive per
neighbour), runs T steps of the FP64 oracle on its extended band, and keeps its own rows.  Each
step spoils one more halo row from the band's cut edge inwards (the oracle applies its boundary
rule there), so after T steps exactly the own rows are still correct.  The assembled result must
equal the oracle on the whole image bit for bit: every pixel goes through the same FP64
operations on the same inputs.  This is the exchange a multi-GPU run of one image would make;
every GPU run of this project is single-GPU, so only the decomposition itself is tested.
"""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys
sys.path.insert(0, os.environ["WMC_ROOT"])
import numpy as np
import torch, torch.distributed as dist
import oracle
from paper_1903_07189_gb300 import synth

rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
h, w, T, iters = int(os.environ["H"]), int(os.environ["W"]), int(os.environ["T"]), int(os.environ["ITERS"])
bnd = os.environ["BND"]
f = synth.make_image(h, w, seed=77, sigma=0.1, dtype=np.float64)
# own rows [a, b): bands as equal as possible
a, b = rank * h // world, (rank + 1) * h // world
lo, hi = max(a - T, 0), min(b + T, h)   # extended band held by this rank
u = f[lo:hi].copy()
for r in range(iters // T):
    # halo exchange: my first / last T own rows to the neighbours above / below
    reqs = []
    if rank > 0:
        reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(u[a - lo:a - lo + T])), rank - 1))
    if rank < world - 1:
        reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(u[b - lo - T:b - lo])), rank + 1))
    if rank > 0:
        top = torch.empty(a - lo, w, dtype=torch.float64)
        dist.recv(top, rank - 1)
        u[:a - lo] = top.numpy()
    if rank < world - 1:
        bot = torch.empty(hi - b, w, dtype=torch.float64)
        dist.recv(bot, rank + 1)
        u[b - lo:] = bot.numpy()
    for q in reqs:
        q.wait()
    u = oracle.denoise(f[lo:hi], 1.0, 0.25, T, bnd, u0=u)
own = np.ascontiguousarray(u[a - lo:b - lo])
np.save(os.path.join(os.environ["OUT"], f"band{rank}.npy"), own)
dist.barrier()
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,bnd", [(2, "replicate"), (3, "zero")])
def test_bands_with_halo_exchange_equal_the_whole_image(tmp_path, world, bnd):
    import oracle
    from paper_1903_07189_gb300 import synth
    h, w, T, iters = 61, 47, 3, 12
    port = free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), WMC_ROOT=ROOT, OUT=str(tmp_path), H=str(h), W=str(w),
                   T=str(T), ITERS=str(iters), BND=bnd)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
    bands = np.concatenate([np.load(tmp_path / f"band{r}.npy") for r in range(world)])
    f = synth.make_image(h, w, seed=77, sigma=0.1, dtype=np.float64)
    whole = oracle.denoise(f, 1.0, 0.25, iters, bnd)
    assert bands.shape == whole.shape
    assert np.array_equal(bands, whole)
