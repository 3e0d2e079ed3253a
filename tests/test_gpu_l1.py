"""L1-fidelity primal-dual iteration (Sec. V-C, A = I) on the GPU against the FP64 oracle.

Per step, from the GPU's own state (U^t, d^t): the dual update d^{t+1} = clip(U^t - f + d^t) has
no neighbours and no selection, so it must match to FP32 rounding; the primal update must lie
within tolerance of U^t + step*(lambda*c - (2 d^{t+1} - d^t)/alpha) for some candidate c in the
tie set of Eq. act (tests/parity_util.py).  Whole trajectories are compared by the fraction of
pixels beyond tolerance and the PSNR between the FP32 and FP64 results.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1903_07189_gb300 import synth
from parity_util import TOL_REL, tie_check, value_range

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
# lambda for [0, 1] images (the L1 term keeps U = f where lambda |H^w| < 1); step / alpha = 0.2 is
# well inside the stable range (< 4/3) of the linearised (U, d) update and step * lambda = 0.5
LAM, STEP, ALPHA = 50.0, 0.01, 0.05


def wmc():
    from paper_1903_07189_gb300 import wmc as m
    return m


def gpu_run(f, iters, u0=None, d=None, boundary="replicate", lam=LAM, step=STEP, alpha=ALPHA):
    out = wmc().denoise_l1(f, lam, step, alpha, iters, boundary, u0=u0, d=d)
    torch.cuda.synchronize()
    return out


def step_check(f64, ut, dt, u1, d1, bnd, lam=LAM, step=STEP, alpha=ALPHA, rows=None, cols=None):
    """Check one GPU step (u1, d1) from (ut, dt); rows/cols restrict the compared window."""
    hw, cand, _ = oracle.wmc_eval(ut, bnd, candidates=True)
    dn = np.clip(ut - f64 + dt, -alpha, alpha)
    R = value_range(ut)
    sl = (slice(None) if rows is None else rows, slice(None) if cols is None else cols)
    assert np.abs(d1[sl] - dn[sl]).max() <= 1e-6 * max(R, alpha)
    transform = lambda c: (ut[sl] + step * (lam * c.transpose(2, 0, 1) - (2 * dn[sl] - dt[sl]) / alpha)).transpose(1, 2, 0)
    ok, ties, err = tie_check(u1[sl], cand[sl], R, transform=transform)
    assert ok.all(), (int((~ok).sum()), err)
    return ties


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
@pytest.mark.parametrize("shape", [(256, 256), (67, 131), (1, 1), (1, 5), (5, 1), (9, 700), (130, 3)])
def test_step_parity(bnd, shape):
    h, w = shape
    f_np = synth.make_image(h, w, seed=h * 1000 + w, sigma=0.1)
    f = torch.from_numpy(f_np).to(DEV)
    d = torch.zeros_like(f)
    ut = gpu_run(f, 5, d=d, boundary=bnd)
    dt = d.clone()
    u1 = gpu_run(f, 1, u0=ut, d=d, boundary=bnd)
    step_check(f_np.astype(np.float64), ut.cpu().double().numpy(), dt.cpu().double().numpy(),
               u1.cpu().double().numpy(), d.cpu().double().numpy(), bnd)


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_trajectory_pr1(bnd):
    """256^2, 8 bumps + 4 shapes, sigma 0.05, 100 iterations: FP32 vs FP64 whole runs."""
    f_np = synth.pr1_image()
    f = torch.from_numpy(f_np).to(DEV)
    d = torch.zeros_like(f)
    u = gpu_run(f, 100, d=d, boundary=bnd).cpu().double().numpy()
    ref, dref = oracle.l1_primal_dual(f_np, LAM, STEP, ALPHA, 100, bnd)
    R = value_range(f_np)
    err = np.abs(u - ref)
    assert (err > TOL_REL * R).mean() <= 1e-3, (err > TOL_REL * R).mean()
    psnr = 10 * np.log10(R * R / np.mean(err ** 2))
    assert psnr >= 80, psnr
    derr = np.abs(d.cpu().double().numpy() - dref)
    assert (derr > TOL_REL * R).mean() <= 1e-3, (derr > TOL_REL * R).mean()


def test_null_d_equals_zero_d_and_resume_is_exact():
    f_np = synth.make_image(90, 77, seed=5, sigma=0.1)
    f = torch.from_numpy(f_np).to(DEV)
    a = gpu_run(f, 9)
    d = torch.zeros_like(f)
    b = gpu_run(f, 9, d=d)
    assert torch.equal(a, b)
    d2 = torch.zeros_like(f)
    u4 = gpu_run(f, 4, d=d2)
    c = gpu_run(f, 5, u0=u4, d=d2)
    assert torch.equal(c, b) and torch.equal(d2, d)


@pytest.mark.parametrize("iters", [1, 2, 5])
def test_in_place_resume(iters):
    f_np = synth.make_image(40, 66, seed=6, sigma=0.1)
    f = torch.from_numpy(f_np).to(DEV)
    d = torch.zeros_like(f)
    u = gpu_run(f, 3, d=d)
    ref_d = d.clone()
    ref = gpu_run(f, iters, u0=u.clone(), d=ref_d)
    out = wmc().denoise_l1(f, LAM, STEP, ALPHA, iters, u0=u, d=d, out=u)
    torch.cuda.synchronize()
    assert torch.equal(out, ref) and torch.equal(d, ref_d)


def test_zero_iterations_and_constant_image():
    f = torch.from_numpy(synth.make_image(30, 20, seed=7)).to(DEV)
    assert torch.equal(gpu_run(f, 0), f)
    c = torch.full((33, 65), 0.25, device=DEV)
    d = torch.zeros_like(c)
    assert torch.equal(gpu_run(c, 12, d=d), c) and torch.count_nonzero(d) == 0


def test_pitched_rows_equal_dense():
    f_np = synth.make_image(50, 61, seed=8, sigma=0.1)
    base = torch.zeros(50, 64, device=DEV)
    base[:, :61] = torch.from_numpy(f_np).to(DEV)
    out = torch.zeros(50, 64, device=DEV)
    d = torch.zeros(50, 64, device=DEV)
    wmc().denoise_l1(base[:, :61], LAM, STEP, ALPHA, 6, d=d[:, :61], out=out[:, :61])
    dense = gpu_run(torch.from_numpy(f_np).to(DEV), 6)
    assert torch.equal(out[:, :61], dense)
    assert torch.count_nonzero(out[:, 61:]) == 0


def test_full_size_sampled_windows():
    """4096^2 (the bench image), 10 iterations then one checked step on windows at the corners,
    the edges and the centre (the oracle evaluates each window on a crop with a 1-pixel margin,
    or the image's own border)."""
    H = W = 4096
    f_np = synth.scale_image(0.02)
    f = torch.from_numpy(f_np).to(DEV)
    d = torch.zeros_like(f)
    ut = gpu_run(f, 10, d=d)
    dt = d.clone()
    u1 = gpu_run(f, 1, u0=ut, d=d)
    ut, dt, u1, d1 = (t.cpu().double().numpy() for t in (ut, dt, u1, d))
    f64 = f_np.astype(np.float64)
    n = 64
    for y0 in (0, H // 2 - n // 2, H - n):
        for x0 in (0, W // 2 - n // 2, W - n):
            ya, yb = max(y0 - 1, 0), min(y0 + n + 1, H)
            xa, xb = max(x0 - 1, 0), min(x0 + n + 1, W)
            rows = slice(y0 - ya, y0 - ya + n)
            cols = slice(x0 - xa, x0 - xa + n)
            crop = lambda a: np.ascontiguousarray(a[ya:yb, xa:xb])
            step_check(crop(f64), crop(ut), crop(dt), crop(u1), crop(d1), "replicate", rows=rows, cols=cols)
