"""The one-launch cluster path for small images (Sec. V-B flow, Eq. MCF): under the default
configuration an image up to 256 x 256 runs all its iterations in one launch of one thread-block
cluster that keeps the image in shared memory.  It must give the bits of the multi-launch path
(same FP32 operations per pixel, same storage rounding) on every shape, dtype and boundary, and
follow the FP64 oracle like it."""
import numpy as np
import pytest
import torch

import oracle
from paper_1903_07189_gb300 import synth
from parity_util import TOL_REL, value_range

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def wmc():
    from paper_1903_07189_gb300 import wmc as m
    return m


def to_gpu(a, dtype=torch.float32, ld=None):
    a = np.asarray(a, dtype=np.float32)
    h, w = a.shape
    if ld is None or ld == w:
        return torch.from_numpy(a).to(DEV).to(dtype)
    buf = torch.full((h, ld), float("nan"), dtype=dtype, device=DEV)
    buf[:, :w] = torch.from_numpy(a).to(dtype)
    return buf[:, :w]


def host(t):
    return t.float().cpu().numpy().astype(np.float64)


def test_cluster_size_rules():
    """ceil(h / 16) CTAs for images up to 256 x 256 and at least two iterations; 0 otherwise.
    Clusters of up to 8 CTAs are portable and must be schedulable on the device."""
    cs = wmc().cluster_size
    for h in (1, 15, 16, 17, 100, 128):
        assert cs(h, 256, 2) == (h + 15) // 16, h
    assert cs(256, 256, 100) in (0, 16)
    assert cs(257, 10, 100) == 0 and cs(10, 257, 100) == 0
    assert cs(100, 100, 1) == 0 and cs(100, 100, 0) == 0
    assert cs(0, 10, 10) == 0 and cs(-1, 10, 10) == 0
    print(f"256 x 256: cluster of {cs(256, 256, 100)} CTAs")


SHAPES = [(1, 1), (2, 2), (1, 256), (256, 1), (16, 16), (17, 33), (96, 80), (128, 256),
          (200, 13), (241, 200), (255, 256), (256, 255), (256, 256)]


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
@pytest.mark.parametrize("shape", SHAPES)
def test_cluster_path_equals_multi_launch_path(shape, bnd):
    """FP32, BF16 and FP16 storage, 2, 3 and 37 iterations: the default (cluster) run equals the
    explicit 4-steps-per-launch run bit for bit."""
    h, w = shape
    img = synth.make_image(h, w, seed=h * 1000 + w, sigma=0.08)
    assert wmc().cluster_size(h, w, 2) > 0 or h > 128
    for dt in (torch.float32, torch.bfloat16, torch.float16):
        f = to_gpu(img, dt)
        for iters in (2, 3, 37):
            got = wmc().denoise(f, 1.0, 0.25, iters, bnd)
            ref = wmc().denoise(f, 1.0, 0.25, iters, bnd, steps_per_launch=4)
            assert torch.equal(got, ref), (dt, iters)


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_cluster_mcf_in_place_and_pitched(bnd):
    """Mean-curvature flow (f None), a run resumed in place (u0 is u) and a pitch that is not a
    multiple of 16 bytes all equal the multi-launch path."""
    img = synth.make_image(150, 211, seed=31, sigma=0.1)
    u0 = to_gpu(img)
    assert torch.equal(wmc().mcf(u0, step=0.3, iters=21, boundary=bnd),
                       wmc().mcf(u0, step=0.3, iters=21, boundary=bnd, steps_per_launch=4))
    f = to_gpu(img)
    full = wmc().denoise(f, 1.5, 0.2, 30, bnd, steps_per_launch=4)
    u = wmc().denoise(f, 1.5, 0.2, 12, bnd)
    wmc().denoise(f, 1.5, 0.2, 18, bnd, u0=u, out=u)
    assert torch.equal(u, full)
    fp = to_gpu(img, ld=213)
    assert torch.equal(wmc().denoise(fp, 1.5, 0.2, 30, bnd), full)


def test_cluster_pr1_graph_and_status():
    """PR1 (eval + 100 iterations) through the cluster path: replayed from a CUDA graph it gives
    the direct call's bits; the call clears a status word that a timed-out wait had set."""
    f = to_gpu(synth.pr1_image())
    ws = torch.empty(wmc().load().wmc_denoise_workspace_size(256, 256, 256, 0), dtype=torch.uint8, device=DEV)
    ref = wmc().denoise(f, 1.0, 0.25, 100, workspace=ws)
    wmc().selftest_wait_timeout(ws, 10_000_000)
    with pytest.raises(wmc().WMCError):
        wmc().check_status(ws)
    out = torch.empty_like(f)
    s = torch.cuda.Stream(DEV)
    s.wait_stream(torch.cuda.current_stream(DEV))
    with torch.cuda.stream(s):
        wmc().denoise(f, 1.0, 0.25, 100, out=out, workspace=ws)
    torch.cuda.current_stream(DEV).wait_stream(s)
    wmc().check_status(ws)
    assert torch.equal(out, ref)
    out.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        wmc().denoise(f, 1.0, 0.25, 100, out=out, workspace=ws)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
@pytest.mark.parametrize("shape", [(256, 256), (200, 13), (33, 250)])
def test_cluster_trajectory_vs_oracle(shape, bnd):
    """25 iterations from the same FP32 input against the FP64 oracle: a selection flip at a
    near-tie moves a pixel by up to step * lambda * 2 |d|, so at most 0.1 % of the pixels may lie
    beyond 1e-5 R."""
    img = synth.make_image(*shape, seed=sum(shape) + 7, sigma=0.05)
    fg = to_gpu(img)
    got = host(wmc().denoise(fg, 1.0, 0.25, 25, bnd))
    want = oracle.denoise(host(fg), 1.0, 0.25, 25, bnd)
    d = np.abs(got - want)
    frac = float((d > TOL_REL * value_range(img)).mean())
    print(f"{shape} {bnd}: max {d.max():.3e} frac>tol {frac:.2e}")
    assert frac <= 1e-3
