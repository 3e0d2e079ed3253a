"""Batched denoising (many images of different sizes, one launch per T-step round) against the
single-image path, which the parity tests tie to the FP64 oracle: every image of a batch must
come out bit-identical to denoising it alone (same FP32 operations per pixel), whatever the
steps per launch, storage type or boundary rule, and a CUDA-graph replay of a run must equal
the direct run."""
import numpy as np
import pytest
import torch

from paper_1903_07189_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

SHAPES = [(1, 1), (3, 200), (97, 31), (250, 130), (64, 64), (131, 257), (5, 7), (300, 9)]


def wmc():
    from paper_1903_07189_gb300 import wmc as m
    return m


def batch_inputs(dtype=torch.float32, shapes=SHAPES, seed=0):
    rng = np.random.default_rng(seed)
    fs = [torch.from_numpy(synth.make_image(h, w, seed=100 + i, sigma=0.08)).to(DEV).to(dtype)
          for i, (h, w) in enumerate(shapes)]
    lams = [float(x) for x in rng.uniform(0.5, 2.0, len(shapes))]
    steps = [0.5 / (1 + l) for l in lams]
    return fs, lams, steps


@pytest.mark.parametrize("tile", [1, 2])
@pytest.mark.parametrize("T", [1, 2, 3, 5, 8])
def test_batch_matches_single_images(T, tile):
    """Both tile shapes (128 x 64 and 128 x 32 regions), every image against itself run alone with
    one step per launch."""
    fs, lams, steps = batch_inputs()
    outs = wmc().denoise_batched(fs, lams, steps, iters=7, steps_per_launch=T, tile=tile)
    for f, l, st, o in zip(fs, lams, steps, outs):
        ref = wmc().denoise(f, l, st, 7, steps_per_launch=1)
        assert torch.equal(o, ref), (f.shape, T, tile)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_batch_reduced_storage_and_zero_boundary(dtype, bnd):
    fs, lams, steps = batch_inputs(dtype, seed=1)
    for tile in (1, 2):
        outs = wmc().denoise_batched(fs, lams, steps, iters=10, boundary=bnd, steps_per_launch=4, tile=tile)
        for f, l, st, o in zip(fs, lams, steps, outs):
            assert torch.equal(o, wmc().denoise(f, l, st, 10, bnd, steps_per_launch=1)), (f.shape, tile)


def test_batch_zero_iterations_copies():
    fs, lams, steps = batch_inputs(seed=2)
    outs = wmc().denoise_batched(fs, lams, steps, iters=0)
    for f, o in zip(fs, outs):
        assert torch.equal(o, f)


def test_batch_pitched_and_shared_input():
    """Pitched rows (no TMA for odd pitches) and two images reading the same f."""
    base = torch.full((70, 129), float("nan"), device=DEV)
    base[:, :101] = torch.from_numpy(synth.make_image(70, 101, seed=3)).to(DEV)
    f = base[:, :101]
    g = torch.from_numpy(synth.make_image(33, 40, seed=4)).to(DEV)
    outs = wmc().denoise_batched([f, f, g], [1.0, 2.0, 0.7], None, iters=9, steps_per_launch=3)
    assert torch.equal(outs[0], wmc().denoise(f, 1.0, None, 9, steps_per_launch=3))
    assert torch.equal(outs[1], wmc().denoise(f, 2.0, None, 9, steps_per_launch=3))
    assert torch.equal(outs[2], wmc().denoise(g, 0.7, None, 9, steps_per_launch=3))


def test_batch_graph_replay_equals_direct_run():
    fs, lams, steps = batch_inputs(seed=5)
    b = wmc().Batch(fs, lams, steps, steps_per_launch=3)
    direct = [o.clone() for o in b.run(11)]
    for o in b.outs:
        o.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run(11)  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.run(11)
    for o in b.outs:
        o.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for d, o in zip(direct, b.outs):
        assert torch.equal(d, o)
    b.check_status()


def test_batch_alias_rejected():
    fs, lams, steps = batch_inputs(shapes=[(40, 50), (40, 50), (40, 50)], seed=6)
    outs = [torch.empty_like(f) for f in fs]
    outs[1] = fs[2]  # writing into another image's input
    with pytest.raises(wmc().WMCError) as e:
        wmc().Batch(fs, lams, steps, outs=outs)
    assert e.value.status == 2


def test_autotune_picks_a_candidate_and_the_plan_matches_single_images():
    """The autotuner times (steps per launch, tile shape) pairs on the caller's batch and returns
    the fastest; a plan with that configuration still gives every image's own bits."""
    fs, lams, steps = batch_inputs(seed=4)
    cands = [(2, 1), (4, 1), (8, 1), (4, 2), (6, 2)]
    best, times = wmc().batch_autotune(fs, lams, steps, candidates=cands, trial_iters=8)
    assert best in cands
    assert all(t > 0 for t in times.values()) and times[best] == min(times.values())
    T, tile = best
    outs = wmc().denoise_batched(fs, lams, steps, iters=9, steps_per_launch=T, tile=tile)
    for f, l, st, o in zip(fs, lams, steps, outs):
        assert torch.equal(o, wmc().denoise(f, l, st, 9, steps_per_launch=T, tile=tile))
    best, times = wmc().batch_autotune(fs, lams, steps, trial_iters=4)  # every default candidate
    assert len(times) == 12 and best in times


def test_batch_rereads_f_on_every_run():
    """Images whose pitch TMA cannot describe (widths that are not a multiple of 4 floats) are read
    from an aligned copy of f in the plan's workspace; the copy is taken at the start of every run,
    so a plan (or a graph of it) follows f when the caller changes it between runs."""
    fs, lams, steps = batch_inputs(shapes=[(70, 101), (33, 40), (65, 130), (9, 7)], seed=7)
    b = wmc().Batch(fs, lams, steps, steps_per_launch=4)
    first = [o.clone() for o in b.run(9)]
    for f, l, st, o in zip(fs, lams, steps, first):
        assert torch.equal(o, wmc().denoise(f, l, st, 9, steps_per_launch=1))
    for f in fs:
        f.mul_(0.5).add_(0.25)
    again = b.run(9)
    for f, l, st, o in zip(fs, lams, steps, again):
        assert torch.equal(o, wmc().denoise(f, l, st, 9, steps_per_launch=1)), f.shape
