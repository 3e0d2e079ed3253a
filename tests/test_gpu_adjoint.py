"""Reverse mode of the unrolled denoising flow (Sec. V-B, A = I) and of the WMC energy
(Eq. wmcr, q = 1) against the FP64 oracle.

The derivative holds each pixel's selection (Eq. act) at its forward value, so the FP32 path and
the FP64 oracle agree only while both pick the same kernel everywhere.  The parity cases below
therefore first check on the oracle's own trajectory that no pixel at any step has a runner-up
candidate within GAP of the winner (a larger gap than FP32 rounding can bridge); under that
condition the gradients must match to FP32 accuracy.  A larger case allows the few pixels that
near-ties touch.  The rest are exact properties: the forward equals wmc_denoise bitwise, results
do not depend on the checkpoint spacing or on the other images of a stack, lambda = 0 has a
closed form, and autograd returns what the C ABI returns.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1903_07189_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GAP = 2e-6  # > 10x the FP32 rounding of a candidate (values in [0, 1], ~30 operations)


def wmc():
    from paper_1903_07189_gb300 import wmc as m
    return m


def image(h, w, seed, sigma=0.05):
    return synth.make_image(h, w, seed=seed, sigma=sigma, dtype=np.float32)


def min_gap(u, bnd):
    """Smallest |runner-up| - |winner| over the pixels of u (FP64 oracle candidates)."""
    _, cand, index = oracle.wmc_eval(u, bnd, candidates=True)
    mag = np.abs(cand)
    win = np.take_along_axis(mag, (index.astype(np.int64) - 1)[..., None], axis=2)[..., 0]
    mag_o = mag.copy()
    np.put_along_axis(mag_o, (index.astype(np.int64) - 1)[..., None], np.inf, axis=2)
    return float((mag_o.min(axis=2) - win).min())


def trajectory_gap(f, lam, step, K, bnd):
    gaps = []
    u = f.astype(np.float64)
    for _ in range(K):
        gaps.append(min_gap(u, bnd))
        u = oracle.denoise(f.astype(np.float64), lam, step, 1, bnd, u0=u)
    return min(gaps)


def gap_map(u, bnd):
    """Per pixel: |runner-up| - |winner| of the FP64 candidates, and the winner's value."""
    hw, cand, index = oracle.wmc_eval(u, bnd, candidates=True)
    mag = np.abs(cand)
    idx = (index.astype(np.int64) - 1)[..., None]
    win = np.take_along_axis(mag, idx, axis=2)[..., 0]
    mag_o = mag.copy()
    np.put_along_axis(mag_o, idx, np.inf, axis=2)
    return mag_o.min(axis=2) - win, hw


def dilate(mask, r):
    """Chebyshev dilation of a boolean image by r pixels."""
    out = mask.copy()
    h, w = mask.shape
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            src = mask[max(-dy, 0):h - max(dy, 0), max(-dx, 0):w - max(dx, 0)]
            out[max(dy, 0):h - max(-dy, 0), max(dx, 0):w - max(-dx, 0)] |= src
    return out


def unrolled_ambiguity(f, lam, step, K, bnd):
    """Pixels of dL/df that a near-tie at some step may touch: a selection at step t enters
    g^t within 1 pixel and reaches grad_f within t + 1 more (one pixel per earlier step)."""
    u = f.astype(np.float64)
    mask = np.zeros(f.shape, dtype=bool)
    for t in range(K):
        gap, _ = gap_map(u, bnd)
        mask |= dilate(gap <= GAP, t + 1)
        u = oracle.denoise(f.astype(np.float64), lam, step, 1, bnd, u0=u)
    return mask


def find_clean_seed(h, w, lam, step, K, bnd, start):
    for seed in range(start, start + 40):
        f = image(h, w, seed)
        if trajectory_gap(f, lam, step, K, bnd) > GAP:
            return seed, f
    raise AssertionError("no seed without near-ties found")


def gpu_grads(fs, lams, step, K, c, bnd, grad_u=None, clean=None):
    f = torch.from_numpy(np.stack(fs)).to(DEV)
    lam = torch.tensor(lams, dtype=torch.float32, device=DEV)
    u, ws = wmc().unrolled_forward(f, lam, step, K, c, bnd)
    if grad_u is None:
        cl = torch.from_numpy(np.stack(clean)).to(DEV)
        n_px = fs[0].size
        grad_u = (2.0 * (u.double() - cl.double()) / n_px).float()
    gf, gl = wmc().unrolled_backward(f, lam, step, K, grad_u, ws, c, bnd)
    torch.cuda.synchronize()
    return u, gf, gl


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
@pytest.mark.parametrize("shape", [(24, 24), (19, 37)])
def test_unrolled_gradient_matches_oracle(bnd, shape):
    h, w = shape
    lam, step, K = 1.0, 0.25, 6
    seed, f = find_clean_seed(h, w, lam, step, K, bnd, start=50)
    clean = synth.make_image(h, w, seed=seed, sigma=0.0, dtype=np.float32)
    loss, dl, df = oracle.unrolled_grad(f, clean, lam, step, K, bnd)
    u, gf, gl = gpu_grads([f], [lam], step, K, 4, bnd, clean=[clean])
    gf = gf[0].cpu().double().numpy()
    assert np.abs(gf - df).max() <= 1e-5 * np.abs(df).max() + 1e-9, (seed, np.abs(gf - df).max())
    assert abs(float(gl[0]) - dl) <= 1e-4 * abs(dl) + 1e-9, (seed, float(gl[0]), dl)
    loss_gpu = float(((u[0].double().cpu().numpy() - clean) ** 2).mean())
    assert abs(loss_gpu - loss) <= 1e-5 * loss


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
@pytest.mark.parametrize("shape", [(70, 140), (97, 65), (5, 150), (150, 5)])
def test_unrolled_gradient_multi_tile(bnd, shape):
    """Several 64 x 32 adjoint tiles with ragged edges: away from the pixels a near-tie can
    touch, dL/df matches to FP32 accuracy; dL/dlambda (a sum over every pixel) to 1e-3."""
    h, w = shape
    lam, step, K = 1.0, 0.25, 4
    f = image(h, w, seed=h + w)
    clean = synth.make_image(h, w, seed=h + w, sigma=0.0, dtype=np.float32)
    mask = unrolled_ambiguity(f, lam, step, K, bnd)
    assert mask.mean() < 0.2, mask.mean()
    loss, dl, df = oracle.unrolled_grad(f, clean, lam, step, K, bnd)
    _, gf, gl = gpu_grads([f], [lam], step, K, 3, bnd, clean=[clean])
    gf = gf[0].cpu().double().numpy()
    err = np.abs(gf - df)[~mask]
    assert err.max() <= 1e-5 * np.abs(df).max() + 1e-9, err.max()
    assert abs(float(gl[0]) - dl) <= 1e-3 * abs(dl), (float(gl[0]), dl)


def test_unrolled_gradient_larger_case_near_ties_local():
    """64 x 80, K = 20: near-ties may flip a selection; away from those the gradient matches."""
    h, w, lam, step, K = 64, 80, 1.5, 0.2, 20
    f = image(h, w, 7, sigma=0.08)
    clean = synth.make_image(h, w, seed=7, sigma=0.0, dtype=np.float32)
    loss, dl, df = oracle.unrolled_grad(f, clean, lam, step, K, "replicate")
    _, gf, gl = gpu_grads([f], [lam], step, K, 7, "replicate", clean=[clean])
    gf = gf[0].cpu().double().numpy()
    err = np.abs(gf - df)
    bad = err > 1e-4 * np.abs(df).max()
    assert bad.mean() <= 0.01, bad.mean()
    assert abs(float(gl[0]) - dl) <= 1e-2 * abs(dl), (float(gl[0]), dl)


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_unrolled_forward_equals_denoise_bitwise(bnd):
    shapes = (45, 67)
    fs = [image(*shapes, seed=s) for s in (1, 2, 3)]
    lams = [0.5, 1.0, 2.0]
    step, K = 0.2, 13
    f = torch.from_numpy(np.stack(fs)).to(DEV)
    lam = torch.tensor(lams, device=DEV)
    for c in (1, 4, 13, 20):
        u, _ = wmc().unrolled_forward(f, lam, step, K, c, bnd)
        for i in range(3):
            ref = wmc().denoise(f[i], lams[i], step, K, bnd)
            assert torch.equal(u[i], ref), (c, i)


def test_checkpoint_spacing_and_stack_invariance():
    h, w = 33, 70
    fs = [image(h, w, seed=s) for s in (11, 12, 13, 14)]
    lams = [0.7, 1.3, 1.0, 2.5]
    step, K = 0.15, 17
    g = torch.from_numpy(np.random.default_rng(5).normal(size=(4, h, w)).astype(np.float32)).to(DEV)
    ref = None
    for c in (1, 2, 5, 17, 40):
        _, gf, gl = gpu_grads(fs, lams, step, K, c, "replicate", grad_u=g)
        if ref is None:
            ref = (gf, gl)
        else:
            assert torch.equal(gf, ref[0]) and torch.equal(gl, ref[1]), c
    for i in range(4):
        _, gf1, gl1 = gpu_grads([fs[i]], [lams[i]], step, K, 5, "replicate", grad_u=g[i:i + 1].contiguous())
        assert torch.equal(gf1[0], ref[0][i]) and torch.equal(gl1[0], ref[1][i]), i


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_lambda_zero_closed_form(bnd):
    """lambda = 0: U^t = f for all t, so dL/df = dL/dU^K and
    dL/dlambda = step * sum_t (1-step)^(K-1-t) <g, H^w(f)>."""
    h, w, step, K = 40, 52, 0.3, 9
    f = image(h, w, seed=21)
    g = np.random.default_rng(8).normal(size=(h, w)).astype(np.float32)
    _, gf, gl = gpu_grads([f], [0.0], step, K, 3, bnd, grad_u=torch.from_numpy(g[None]).to(DEV))
    np.testing.assert_allclose(gf[0].cpu().numpy(), g, rtol=1e-5, atol=1e-6)
    hw = oracle.wmc_eval(f.astype(np.float64), bnd)
    expect = step * sum((1 - step) ** (K - 1 - t) for t in range(K)) * float((g.astype(np.float64) * hw).sum())
    assert abs(float(gl[0]) - expect) <= 1e-4 * abs(expect)


def test_zero_steps():
    f = image(20, 30, seed=4)
    g = np.random.default_rng(9).normal(size=(1, 20, 30)).astype(np.float32)
    u, gf, gl = gpu_grads([f], [1.0], 0.25, 0, 3, "replicate", grad_u=torch.from_numpy(g).to(DEV))
    assert torch.equal(u[0].cpu(), torch.from_numpy(f))
    assert torch.equal(gf.cpu(), torch.from_numpy(g))
    assert float(gl[0]) == 0.0


def test_autograd_function_matches_abi_and_finite_difference():
    h, w, step, K = 48, 40, 0.25, 10
    f_np = image(h, w, seed=31, sigma=0.08)
    clean = torch.from_numpy(synth.make_image(h, w, seed=31, sigma=0.0, dtype=np.float32)).to(DEV)
    f = torch.from_numpy(f_np).to(DEV).requires_grad_(True)
    lam = torch.tensor([1.2], device=DEV, requires_grad=True)
    u = wmc().unrolled_denoise(f, lam, step, K, ckpt_every=3)
    loss = ((u - clean) ** 2).mean()
    loss.backward()
    _, gf, gl = gpu_grads([f_np], [1.2], step, K, 3, "replicate", clean=[clean.cpu().numpy()])
    assert torch.allclose(f.grad, gf[0], rtol=1e-5, atol=1e-9)
    assert torch.allclose(lam.grad, gl, rtol=1e-5)

    def L(lv):
        with torch.no_grad():
            uu = wmc().unrolled_denoise(f.detach(), torch.tensor([lv], device=DEV), step, K)
            return float(((uu.double() - clean.double()) ** 2).mean())
    eps = 1e-3
    fd = (L(1.2 + eps) - L(1.2 - eps)) / (2 * eps)
    assert abs(fd - float(lam.grad)) <= 0.05 * abs(fd) + 1e-8, (fd, float(lam.grad))


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
@pytest.mark.parametrize("shape", [(30, 30), (17, 45), (100, 200), (257, 131)])
def test_energy_grad_matches_oracle(bnd, shape):
    """Exact (FP32 rounding) wherever no pixel next to q has a near-tie or a near-zero H^w."""
    u = image(*shape, seed=200 + shape[0])
    u64 = u.astype(np.float64)
    gap, hw = gap_map(u64, bnd)
    mask = dilate((gap <= GAP) | (np.abs(hw) <= GAP), 1)
    assert mask.mean() < 0.05, mask.mean()
    ref = oracle.energy_grad(u64, bnd)
    got = wmc().energy_grad(torch.from_numpy(u).to(DEV), bnd).cpu().double().numpy()
    np.testing.assert_allclose(got[~mask], ref[~mask], rtol=0, atol=1e-6)


@pytest.mark.parametrize("bnd,shape", [(b, s) for b in ("replicate", "zero")
                                       for s in [(2, 2), (3, 65), (2, 130), (33, 2), (65, 3)]]
                         + [("replicate", (1, 70)), ("replicate", (70, 1))])
def test_energy_grad_thin_images(bnd, shape):
    """A few rows or columns: every pixel is a border pixel, so the REPLICATE fold of the ring
    terms (top and bottom, left and right on the same pixel) is exercised everywhere.  (One-row
    images are mostly ties: a row's vertical neighbours are its own values or zeros; under ZERO
    every pixel is one.)"""
    u = image(*shape, seed=300 + shape[0] + shape[1])
    u64 = u.astype(np.float64)
    gap, hw = gap_map(u64, bnd)
    mask = dilate((gap <= GAP) | (np.abs(hw) <= GAP), 1)
    assert (~mask).sum() >= min(10, mask.size), mask.mean()
    ref = oracle.energy_grad(u64, bnd)
    got = wmc().energy_grad(torch.from_numpy(u).to(DEV), bnd).cpu().double().numpy()
    np.testing.assert_allclose(got[~mask], ref[~mask], rtol=0, atol=1e-6)


def test_energy_grad_constant_image_is_zero():
    u = torch.full((25, 31), 0.375, device=DEV)
    assert torch.count_nonzero(wmc().energy_grad(u)) == 0


def test_energy_grad_pitched_rows():
    base = torch.zeros(40, 64, device=DEV)
    u_np = image(40, 50, seed=222)
    base[:, :50] = torch.from_numpy(u_np).to(DEV)
    got = wmc().energy_grad(base[:, :50]).cpu().double().numpy()
    dense = wmc().energy_grad(torch.from_numpy(u_np).to(DEV)).cpu().double().numpy()
    assert np.array_equal(got, dense)


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_one_call_backward_equals_the_two_unrolled_calls(bnd):
    """wmc_backward (forward sweep with checkpoints, then the reverse sweep, in one call) gives the
    bits of wmc_unrolled_forward followed by wmc_unrolled_backward."""
    h, w, step, K, c = 45, 131, 0.2, 11, 4
    f = torch.from_numpy(np.stack([image(h, w, seed=s) for s in (31, 32, 33)])).to(DEV)
    lam = torch.tensor([0.6, 1.1, 1.9], device=DEV)
    g = torch.from_numpy(np.random.default_rng(12).normal(size=(3, h, w)).astype(np.float32)).to(DEV)
    _, ws = wmc().unrolled_forward(f, lam, step, K, c, bnd)
    gf, gl = wmc().unrolled_backward(f, lam, step, K, g, ws, c, bnd)
    gf1, gl1 = wmc().backward(f, lam, step, K, g, c, bnd)
    assert torch.equal(gf1, gf) and torch.equal(gl1, gl)
