"""The workloads' full sizes, in the launch configurations the benchmark times.

- precision: a 16384 x 16384 image stored as FP32, BF16 and FP16; after 5 steps one more step is
  checked at sampled pixels against the oracle's point-wise step (tie excusal; for 16-bit storage
  half an ulp of the stored result on top);
- batch: the 512 uneven images (sides 64..1536), one 4-step launch per round; sampled images must
  equal the single-image path bit for bit, and one image's step is checked against the oracle;
- scale: the 4096 x 4096 image after 20 iterations; its FP64 energies (the last kernel of every
  benchmark step) against the oracle's;
- diff: 32 images of 512 x 512, K = 50, checkpoints every 7: the forward equals wmc_denoise bit
  for bit, the gradients do not depend on the checkpoint spacing, and dL/dlambda agrees with a
  central difference of the loss.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1903_07189_gb300 import synth
from parity_util import tie_check, value_range

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def wmc():
    from paper_1903_07189_gb300 import wmc as m
    return m


def host(t):
    return t.float().cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def precision_image():
    return synth.make_image(16384, 16384, seed=3, n_bumps=64, n_shapes=32, sigma=0.05)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
def test_precision_config_sampled_step(precision_image, dtype):
    n = 16384
    f = torch.from_numpy(precision_image).to(DEV).to(dtype)
    ut = wmc().denoise(f, 1.0, 0.25, 5)
    u1 = wmc().denoise(f, 1.0, 0.25, 1, u0=ut)
    rng = np.random.default_rng(31)
    ys = np.concatenate([[0, 0, n - 1, n - 1], rng.integers(0, n, 1996)])
    xs = np.concatenate([[0, n - 1, 0, n - 1], rng.integers(0, n, 1996)])
    yt = torch.from_numpy(ys).to(DEV)
    xt = torch.from_numpy(xs).to(DEV)
    # the oracle needs each sampled pixel's 3x3 neighbourhood of U^t: gather 3x3 patches
    U = ut.float()
    patches = np.zeros((ys.size, 3, 3))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            yy = (yt + dy).clamp(0, n - 1)
            xx = (xt + dx).clamp(0, n - 1)
            patches[:, dy + 1, dx + 1] = U[yy, xx].cpu().numpy()
    cand = np.stack([oracle.eval_points(p, [1], [1], candidates=True)[1][0] for p in patches])
    Up = patches[:, 1, 1]
    fp = f.float()[yt, xt].cpu().numpy().astype(np.float64)
    got = u1.float()[yt, xt].cpu().numpy().astype(np.float64)
    tr = lambda c: Up[:, None] + 0.25 * (c - (Up[:, None] - fp[:, None]))
    extra = None
    if dtype != torch.float32:
        ulp = {torch.bfloat16: 2.0 ** -8, torch.float16: 2.0 ** -11}[dtype]
        extra = np.abs(got) * ulp
    ok, _, err = tie_check(got, cand, value_range(precision_image), transform=tr, extra_tol=extra)
    assert ok.all(), err


def test_batch_config_matches_single_images_and_oracle():
    n = 512
    sizes = synth.batch_sizes(n)
    params = synth.batch_params(n)
    fs = [torch.from_numpy(synth.make_image(h, w, seed=1000 + i, n_bumps=8, n_shapes=4, sigma=sg)).to(DEV)
          for i, ((h, w), (sg, _)) in enumerate(zip(sizes, params))]
    lams = [l for _, l in params]
    steps = [0.5 / (1 + l) for l in lams]
    outs = wmc().denoise_batched(fs, lams, steps, iters=8, steps_per_launch=4)
    rng = np.random.default_rng(7)
    for i in rng.choice(n, 16, replace=False):
        ref = wmc().denoise(fs[i], lams[i], steps[i], 8, steps_per_launch=4)
        assert torch.equal(outs[i], ref), i
    # one image: step 9 from the batch's U^8 against the oracle
    i = int(rng.integers(n))
    u9 = wmc().denoise(fs[i], lams[i], steps[i], 1, u0=outs[i])
    U, F = host(outs[i]), host(fs[i])
    _, cand, _ = oracle.wmc_eval(U, candidates=True)
    tr = lambda c: U[..., None] + steps[i] * (lams[i] * c - (U[..., None] - F[..., None]))
    ok, _, err = tie_check(host(u9), cand, value_range(U), transform=tr)
    assert ok.all(), (i, err)


def test_diff_config_properties():
    n, h, w, K, step = 32, 512, 512, 50, 0.25
    pairs = [synth.make_image(h, w, seed=2000 + i, n_bumps=8, n_shapes=4, sigma=0.05, return_clean=True)
             for i in range(n)]
    f = torch.from_numpy(np.stack([p[0] for p in pairs])).to(DEV)
    clean = torch.from_numpy(np.stack([p[1] for p in pairs])).to(DEV)
    lam = torch.full((n,), 1.0, device=DEV)
    u, ws = wmc().unrolled_forward(f, lam, step, K, 7)
    for i in (0, 17):
        assert torch.equal(u[i], wmc().denoise(f[i], 1.0, step, K)), i
    g = (2.0 * (u.double() - clean.double()) / u.numel()).float()
    gf7, gl7 = wmc().unrolled_backward(f, lam, step, K, g, ws, 7)
    u50, ws50 = wmc().unrolled_forward(f, lam, step, K, 50)
    gf50, gl50 = wmc().unrolled_backward(f, lam, step, K, g, ws50, 50)
    assert torch.equal(u50, u) and torch.equal(gf7, gf50) and torch.equal(gl7, gl50)

    def loss(lv):
        uu, _ = wmc().unrolled_forward(f, lv, step, K, 7)
        return float(((uu.double() - clean.double()) ** 2).mean())
    eps = 1e-3
    for i in (3, 29):
        e = torch.zeros(n, device=DEV)
        e[i] = eps
        fd = (loss(lam + e) - loss(lam - e)) / (2 * eps)
        assert abs(fd - float(gl7[i])) <= 0.05 * abs(fd) + 1e-9, (i, fd, float(gl7[i]))


def test_scale_config_energies():
    f = torch.from_numpy(synth.make_image(4096, 4096, seed=1, n_bumps=64, n_shapes=32, sigma=0.02)).to(DEV)
    u = wmc().denoise(f, 1.0, 0.25, 20)
    e = wmc().energy(u, f).cpu().numpy()
    want = oracle.energies(host(u), host(f))
    np.testing.assert_allclose(e[:2], want[:2], rtol=1e-6)
    assert e[2] == 0.0 and np.array_equal(e, wmc().energy(u, f).cpu().numpy())
