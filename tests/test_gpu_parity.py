"""GPU parity: libwmc.so (through the C ABI) against the FP64 oracle on the same seeded inputs.

Eval (Sec. IV-B, Eq. conv / Eq. act) is compared pixel by pixel with tie excusal; the flow
(Sec. V-B, Eq. MCF) is compared one Jacobi step at a time from the GPU's own U^t (a flip of
the selection at a near-tie makes long trajectories diverge locally, so per-step parity is
the gate and whole-trajectory differences are checked against a looser bound and reported).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1903_07189_gb300 import synth
from parity_util import TOL_REL, tie_check, value_range

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


def eval_parity(u32, bnd, ld=None, dtype=torch.float32):
    ug = to_gpu(u32, dtype, ld)
    uin = host(ug)  # exactly what the GPU read
    hw = wmc().eval(ug, bnd)
    torch.cuda.synchronize()
    _, cand, _ = oracle.wmc_eval(uin, bnd, candidates=True)
    R = value_range(uin)
    extra = None
    if dtype != torch.float32:
        # output rounded to storage: half an ulp of the stored value
        ulp = {torch.bfloat16: 2.0 ** -8, torch.float16: 2.0 ** -11}[dtype]
        extra = np.abs(host(hw)) * ulp + 1e-30
    ok, ties, err = tie_check(host(hw), cand, R, extra_tol=extra)
    return ok, ties, err


SHAPES = [(1, 1), (1, 9), (7, 1), (2, 2), (3, 5), (64, 64), (63, 65), (67, 129), (130, 61), (200, 333)]


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
@pytest.mark.parametrize("shape", SHAPES)
def test_eval_parity_shapes(shape, bnd):
    u = synth.make_image(*shape, seed=sum(shape), sigma=0.05)
    ok, ties, err = eval_parity(u, bnd)
    assert ok.all(), (err, np.argwhere(~ok)[:5])


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_eval_parity_pitched(bnd):
    u = synth.make_image(61, 70, seed=3, sigma=0.05)
    ok, _, err = eval_parity(u, bnd, ld=96)
    assert ok.all(), err


def test_eval_parity_pr1_image():
    """256 x 256, 8 bumps + 4 shapes, sigma 0.05, seed 0 (the small reference workload)."""
    u = synth.pr1_image()
    for bnd in ["replicate", "zero"]:
        ok, ties, err = eval_parity(u, bnd)
        assert ok.all(), (bnd, err)


def test_eval_parity_structured_images():
    """Ramps (exact opposite-sign ties everywhere), steps, integer images."""
    y, x = np.mgrid[0:40, 0:50].astype(np.float64)
    for u in [x + 2 * y, 3 * x - y, (x >= 20) * 1.0, (x + y >= 30) * 1.0, x ** 2 / 100,
              np.random.default_rng(0).integers(0, 5, (40, 50)).astype(np.float64)]:
        ok, _, err = eval_parity(u.astype(np.float32), "replicate")
        assert ok.all(), err


@pytest.mark.parametrize("shape", [(64, 128), (65, 129), (200, 517), (3, 700), (1000, 130), (7, 5)])
@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_eval_tma_path_equals_streaming_path(shape, bnd):
    """Dense FP32 rows (16-byte aligned) are evaluated by the persistent TMA kernel, an odd pitch
    takes the streaming kernel: both must give the same bits (ragged boxes, both boundaries,
    images smaller than one box), and the evaluation status word stays clear."""
    u = synth.make_image(*shape, seed=26, sigma=0.07)
    dense = to_gpu(u)
    pitched = to_gpu(u, ld=shape[1] + 1)
    a = wmc().eval(dense, bnd)
    b = wmc().eval(pitched, bnd)
    assert torch.equal(a, b)
    ok, _, err = eval_parity(u, bnd)
    assert ok.all(), err
    wmc().eval_status()


@pytest.mark.parametrize("R", [16, 64])
def test_smooth_disk_eval_and_energy(R):
    """Smooth disks (edge width R/4; the gradient turns through every direction, so every
    selection branch and the 8-direction axis bias are exercised): evaluation against the oracle
    with tie excusal, and the FP64 energy sum |H^w| within 2e-6."""
    n = int(2 * R * 1.75) + 8
    c = (n - 1) / 2.0
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    u = (0.5 * (1 + np.tanh((R - np.hypot(y - c, x - c)) / (0.25 * R)))).astype(np.float32)
    for bnd in ("replicate", "zero"):
        ok, _, err = eval_parity(u, bnd)
        assert ok.all(), (bnd, err)
        e = float(wmc().energy(to_gpu(u), boundary=bnd)[0])
        want = oracle.energies(u.astype(np.float64), boundary=bnd)[0]
        assert abs(e - want) <= 2e-6 * abs(want), (bnd, e, want)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_eval_parity_reduced_storage(dtype):
    u = synth.make_image(97, 131, seed=11, sigma=0.05)
    ok, _, err = eval_parity(u, "replicate", dtype=dtype)
    assert ok.all(), err


def test_eval_full_size_sampled():
    """4096 x 4096 (64 bumps, 32 shapes, sigma 0.02): 40000 random pixels plus the border."""
    u = synth.scale_image(0.02)
    ug = to_gpu(u)
    hw = host(wmc().eval(ug))
    uin = u.astype(np.float64)
    rng = np.random.default_rng(5)
    n = 40000
    ys = np.concatenate([rng.integers(0, 4096, n), np.zeros(512, int), np.full(512, 4095),
                         rng.integers(0, 4096, 1024)])
    xs = np.concatenate([rng.integers(0, 4096, n), rng.integers(0, 4096, 1024),
                         np.r_[np.zeros(512, int), np.full(512, 4095)]])
    _, cand = oracle.eval_points(uin, ys, xs, candidates=True)
    ok, _, err = tie_check(hw[ys, xs], cand, value_range(uin))
    assert ok.all(), err


# --------------------------------------------------------------------------- flows
def step_parity(f32, lam, step, bnd, t_list, mcf=False, size_tag=""):
    """GPU U^t, then one more GPU step, vs the oracle's step from the GPU's own U^t."""
    fg = to_gpu(f32)
    fin = host(fg)
    R = value_range(fin)
    for t in t_list:
        if mcf:
            ut = wmc().mcf(fg, step=step, iters=t, boundary=bnd)
            ut1 = wmc().mcf(ut, step=step, iters=1, boundary=bnd)
        else:
            ut = wmc().denoise(fg, lam, step, t, bnd)
            ut1 = wmc().denoise(fg, lam, step, 1, bnd, u0=ut)
        U = host(ut)
        _, cand, _ = oracle.wmc_eval(U, bnd, candidates=True)
        mu = 0.0 if mcf else 1.0
        tr = lambda c: U[..., None] + step * (lam * c - mu * (U[..., None] - fin[..., None]))
        ok, ties, err = tie_check(host(ut1), cand, R, transform=tr)
        assert ok.all(), (size_tag, t, err)


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_denoise_step_parity_pr1(bnd):
    step_parity(synth.pr1_image(), 1.0, 0.25, bnd, [0, 1, 10, 50, 99])


@pytest.mark.parametrize("shape", [(1, 1), (1, 40), (33, 1), (5, 7), (67, 129), (131, 70)])
def test_denoise_step_parity_shapes(shape):
    step_parity(synth.make_image(*shape, seed=13, sigma=0.08), 1.5, 0.2, "replicate", [0, 3, 9],
                size_tag=shape)


def test_mcf_step_parity():
    step_parity(synth.make_image(90, 120, seed=14), 1.0, 0.4, "replicate", [0, 5, 20], mcf=True)


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_steps_per_launch_bitwise_invariant(bnd):
    """T Jacobi steps in shared memory per launch give bit-identical results for T = 1..8
    (every configuration performs the same FP32 operations per pixel)."""
    f = to_gpu(synth.make_image(150, 173, seed=15, sigma=0.1))
    ref = wmc().denoise(f, 1.0, 0.25, 17, bnd, steps_per_launch=1)
    for tile in (1, 2):
        for T in range(2, 9):
            got = wmc().denoise(f, 1.0, 0.25, 17, bnd, steps_per_launch=T, tile=tile)
            assert torch.equal(got, ref), (T, tile)


def test_pr1_trajectory_vs_oracle():
    """100 iterations, lambda 1, step 0.25, replicate: the whole FP32 trajectory against the
    FP64 oracle from the same FP32 input.  Selection flips at near-ties make isolated pixels
    differ by up to step*lambda*2|d|, so the gate is: at most 0.1% of the pixels beyond
    1e-5 R, and the two results within 80 dB PSNR of each other."""
    f = synth.pr1_image()
    fg = to_gpu(f)
    got = host(wmc().denoise(fg, 1.0, 0.25, 100))
    want = oracle.denoise(host(fg), 1.0, 0.25, 100)
    R = value_range(f)
    d = np.abs(got - want)
    frac = float((d > TOL_REL * R).mean())
    mse = float((d ** 2).mean())
    psnr = 10 * np.log10(R * R / mse) if mse > 0 else np.inf
    print(f"PR1 trajectory: max {d.max():.3e}  p99.99 {np.quantile(d, 0.9999):.3e}  "
          f"frac>tol {frac:.2e}  psnr {psnr:.1f} dB")
    assert frac <= 1e-3
    assert psnr >= 80


def test_denoise_full_size_sampled_step():
    """4096 x 4096: U^7 on the GPU (T = 4: one full launch + a 3-step remainder), then one more
    step, checked at 40000 sampled pixels against the oracle's point-wise step."""
    f = synth.scale_image(0.1)
    fg = to_gpu(f)
    ut = wmc().denoise(fg, 1.0, 0.25, 7)
    ut1 = host(wmc().denoise(fg, 1.0, 0.25, 1, u0=ut))
    U = host(ut)
    rng = np.random.default_rng(6)
    ys = np.concatenate([rng.integers(0, 4096, 40000), [0, 0, 4095, 4095]])
    xs = np.concatenate([rng.integers(0, 4096, 40000), [0, 4095, 0, 4095]])
    _, cand = oracle.eval_points(U, ys, xs, candidates=True)
    Up, fp = U[ys, xs], f.astype(np.float64)[ys, xs]
    tr = lambda c: Up[:, None] + 0.25 * (1.0 * c - (Up[:, None] - fp[:, None]))
    ok, _, err = tie_check(ut1[ys, xs], cand, value_range(f), transform=tr)
    assert ok.all(), err


def test_full_size_properties():
    """4096 x 4096, 20 steps: max principle (step (1 + lambda) <= 1), exact contrast
    homogeneity for alpha = 2 and -0.5, run-to-run determinism."""
    f = to_gpu(synth.scale_image(0.1))
    u = wmc().denoise(f, 1.0, 0.25, 20)
    assert float(u.min()) >= float(f.min()) and float(u.max()) <= float(f.max())
    assert torch.equal(wmc().denoise(f, 1.0, 0.25, 20), u)
    assert torch.equal(wmc().denoise(2 * f, 1.0, 0.25, 20), 2 * u)
    assert torch.equal(wmc().denoise(-0.5 * f, 1.0, 0.25, 20), -0.5 * u)


def test_resume_and_in_place():
    f = to_gpu(synth.make_image(77, 91, seed=16))
    full = wmc().denoise(f, 1.0, 0.25, 13)
    part = wmc().denoise(f, 1.0, 0.25, 6)
    rest = wmc().denoise(f, 1.0, 0.25, 7, u0=part)
    assert torch.equal(rest, full)
    # in place: u0 is u (odd and even launch counts, exercising the copy-back path)
    for a, b in [(6, 7), (4, 9), (5, 8)]:
        u = wmc().denoise(f, 1.0, 0.25, a)
        wmc().denoise(f, 1.0, 0.25, b, u0=u, out=u)
        assert torch.equal(u, full), (a, b)


def test_zero_iterations_copies():
    f = to_gpu(synth.make_image(20, 30, seed=17))
    assert torch.equal(wmc().denoise(f, 1.0, 0.25, 0), f)


def test_energy_parity():
    f, clean = synth.make_image(300, 217, seed=18, sigma=0.1, return_clean=True)
    fg, cg = to_gpu(f), to_gpu(clean)
    ug = wmc().denoise(fg, 1.0, 0.25, 10)
    e = wmc().energy(ug, fg, cg).cpu().numpy()
    want = oracle.energies(host(ug), host(fg), host(cg))
    np.testing.assert_allclose(e, want, rtol=2e-6)
    e2 = wmc().energy(ug, fg, cg).cpu().numpy()
    assert np.array_equal(e, e2)  # fixed summation order


@pytest.mark.parametrize("shape,ld", [((301, 1300), None), ((70, 133), 136), ((5, 4), None), ((2, 2049), 2052),
                                      ((33, 218), None), ((19, 131), 133)])
@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_energy_layouts(shape, ld, bnd):
    """FP32 rows that are 16-byte aligned take the TMA-fed energy kernel, the rest the streaming
    kernels; ragged widths and heights, NaN-filled pitch padding (never read), and every
    combination of the optional f / clean terms (each a separate kernel instance with its own
    box offsets) must match the oracle and repeat bitwise."""
    f, clean = synth.make_image(*shape, seed=23, sigma=0.1, return_clean=True)
    fg, cg = to_gpu(f, ld=ld), to_gpu(clean, ld=ld)
    ug = wmc().denoise(fg, 1.0, 0.25, 3, boundary=bnd)
    U = host(ug)
    for args, want in [((ug, fg, cg), oracle.energies(U, host(fg), host(cg), boundary=bnd)),
                       ((ug, fg, None), oracle.energies(U, host(fg), None, boundary=bnd)),
                       ((ug, None, cg), oracle.energies(U, None, host(cg), boundary=bnd)),
                       ((ug, None, None), oracle.energies(U, None, None, boundary=bnd))]:
        e = wmc().energy(*args, boundary=bnd).cpu().numpy()
        np.testing.assert_allclose(e, want, rtol=2e-6, atol=1e-300)
        assert np.array_equal(e, wmc().energy(*args, boundary=bnd).cpu().numpy())


def test_host_entry_point_matches_device():
    f = synth.make_image(129, 257, seed=19)
    fh = torch.from_numpy(f).pin_memory()
    out = wmc().denoise_host(fh, 1.0, 0.25, 11)
    torch.cuda.synchronize()
    ref = wmc().denoise(torch.from_numpy(f).to(DEV), 1.0, 0.25, 11).cpu()
    assert torch.equal(out, ref)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_reduced_storage_step(dtype):
    """One step with BF16/FP16 storage: FP32 arithmetic on the widened inputs, then one
    round-to-nearest-even store; within half an ulp of the stored value of the oracle step."""
    f = to_gpu(synth.make_image(111, 97, seed=20, sigma=0.05), dtype)
    u1 = wmc().denoise(f, 1.0, 0.25, 1)
    F = host(f)
    _, cand, _ = oracle.wmc_eval(F, candidates=True)
    ulp = {torch.bfloat16: 2.0 ** -8, torch.float16: 2.0 ** -11}[dtype]
    g = host(u1)
    tr = lambda c: F[..., None] + 0.25 * c
    ok, _, err = tie_check(g, cand, value_range(F), transform=tr, extra_tol=np.abs(g) * ulp)
    assert ok.all(), err


@pytest.mark.parametrize("shape,ld", [((61, 61), None), ((70, 133), 135), ((129, 250), 256), ((3, 200), None)])
def test_flow_pitches_and_fallbacks(shape, ld):
    """Odd widths / pitches take the plain-load path of the multi-step kernel (no TMA: the row
    pitch is not a multiple of 16 bytes) and the unpaired-column paths; results must still be
    bit-identical across steps_per_launch and match the oracle step by step."""
    f32 = synth.make_image(*shape, seed=21, sigma=0.07)
    fg = to_gpu(f32, ld=ld)
    ref = wmc().denoise(fg, 1.0, 0.25, 9, steps_per_launch=1)
    for T in (2, 3, 5, 8):
        assert torch.equal(wmc().denoise(fg, 1.0, 0.25, 9, steps_per_launch=T), ref), T
    U = host(wmc().denoise(fg, 1.0, 0.25, 8, steps_per_launch=4))
    u9 = host(wmc().denoise(fg, 1.0, 0.25, 1, u0=to_gpu(U.astype(np.float32), ld=ld)))
    _, cand, _ = oracle.wmc_eval(U, candidates=True)
    F = host(fg)
    tr = lambda c: U[..., None] + 0.25 * (c - (U[..., None] - F[..., None]))
    ok, _, err = tie_check(u9, cand, value_range(F), transform=tr)
    assert ok.all(), err


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_reduced_storage_steps_per_launch_bitwise(dtype, bnd):
    """Every step rounds to the storage type, inside a multi-step launch too, so T = 1..8 agree
    bit for bit for BF16/FP16 as well."""
    f = to_gpu(synth.make_image(140, 301, seed=22, sigma=0.1), dtype)
    ref = wmc().denoise(f, 1.0, 0.25, 11, bnd, steps_per_launch=1)
    for T in range(2, 9):
        assert torch.equal(wmc().denoise(f, 1.0, 0.25, 11, bnd, steps_per_launch=T), ref), T


def test_status_word_ok_after_runs():
    f = to_gpu(synth.make_image(300, 300, seed=23))
    ws = torch.empty(wmc().load().wmc_denoise_workspace_size(300, 300, 300, 0), dtype=torch.uint8, device=DEV)
    wmc().denoise(f, 1.0, 0.25, 12, steps_per_launch=4, workspace=ws)
    wmc().check_status(ws)  # raises on WMC_ERR_TIMEOUT


def test_timed_out_wait_is_reported_and_the_context_stays_usable():
    """A bounded wait that runs out (the self-test's mbarrier is armed for a transfer that is
    never issued; 10 ms limit) sets the status word: check_status raises WMC_ERR_TIMEOUT.  The
    next flow call on the workspace clears the word, and its result is still exact."""
    f = to_gpu(synth.make_image(150, 170, seed=25))
    ws = torch.empty(wmc().load().wmc_denoise_workspace_size(150, 170, 170, 0), dtype=torch.uint8, device=DEV)
    ref = wmc().denoise(f, 1.0, 0.25, 8, steps_per_launch=4, workspace=ws)
    wmc().check_status(ws)
    wmc().selftest_wait_timeout(ws, 10_000_000)
    with pytest.raises(wmc().WMCError) as err:
        wmc().check_status(ws)
    assert err.value.status == 5  # WMC_ERR_TIMEOUT
    again = wmc().denoise(f, 1.0, 0.25, 8, steps_per_launch=4, workspace=ws)
    wmc().check_status(ws)
    assert torch.equal(again, ref)


def test_eval_timeout_is_reported_once_and_cleared():
    """The evaluation status word (set when a bounded TMA wait of the persistent evaluation
    kernel runs out) is made to read WMC_ERR_TIMEOUT by the self-test's wait that nothing
    completes (10 ms); wmc_eval_status reports it once and clears it, and evaluation still gives
    the exact result afterwards."""
    u = to_gpu(synth.make_image(130, 260, seed=27))
    ref = wmc().eval(u)
    wmc().eval_status()
    wmc().selftest_status_timeout("eval", 10_000_000)
    with pytest.raises(wmc().WMCError) as err:
        wmc().eval_status()
    assert err.value.status == 5  # WMC_ERR_TIMEOUT
    wmc().eval_status()  # cleared by the previous read
    assert torch.equal(wmc().eval(u), ref)
    wmc().eval_status()


def test_mcf_steps_per_launch_bitwise():
    u0 = to_gpu(synth.make_image(200, 180, seed=24))
    ref = wmc().mcf(u0, step=0.3, iters=10, steps_per_launch=1)
    for T in (2, 4, 7):
        assert torch.equal(wmc().mcf(u0, step=0.3, iters=10, steps_per_launch=T), ref), T


def test_denoise_graph_capture_replay():
    """A single-image run (consecutive tile launches chained as programmatic dependents) captured
    into a CUDA graph replays to the same bits as the direct call."""
    f = to_gpu(synth.make_image(300, 260, seed=23, sigma=0.1))
    out = torch.empty_like(f)
    ws = torch.empty(wmc().load().wmc_denoise_workspace_size(300, 260, 260, 0), dtype=torch.uint8,
                     device=DEV)
    ref = wmc().denoise(f, 1.0, 0.25, 18, out=torch.empty_like(f), workspace=ws)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        wmc().denoise(f, 1.0, 0.25, 18, out=out, workspace=ws)  # warm-up off the capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        wmc().denoise(f, 1.0, 0.25, 18, out=out, workspace=ws)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
@pytest.mark.parametrize("shape", [(59, 123), (117, 245), (51, 115), (27, 123), (53, 245), (175, 65),
                                   (3, 130), (130, 3), (61, 61), (1, 1), (1, 200), (200, 1), (2, 300)])
def test_overhanging_tiles_bitwise_invariant(bnd, shape):
    """Images one cell past a whole number of output tiles (128 x 64 regions: 122 x 58 at T = 4,
    114 x 50 at T = 8; 128 x 32 regions: 122 x 26 at T = 4), where the last tile row or column
    overhangs the image and its outer warps skip work, and images one or two cells high or wide,
    whose border tiles compute every cell from a clamped column or store it into a ring row: every
    T and tile shape still gives the one-step-per-launch bits."""
    f = to_gpu(synth.make_image(*shape, seed=sum(shape), sigma=0.1))
    ref = wmc().denoise(f, 1.0, 0.25, 11, bnd, steps_per_launch=1)
    for tile in (1, 2):
        for T in (2, 4, 5, 8):
            assert torch.equal(wmc().denoise(f, 1.0, 0.25, 11, bnd, steps_per_launch=T, tile=tile), ref), (T, tile)
    bf = f.to(torch.bfloat16)
    ref16 = wmc().denoise(bf, 1.0, 0.25, 11, bnd, steps_per_launch=1)
    for tile in (1, 2):
        assert torch.equal(wmc().denoise(bf, 1.0, 0.25, 11, bnd, steps_per_launch=4, tile=tile), ref16)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("iters", [5, 8, 13])
def test_unaligned_pitch_is_staged_bit_exactly(dtype, iters):
    """Rows whose pitch is not a multiple of 16 bytes (TMA cannot describe them) are staged through
    aligned workspace images for the multi-step launches; the result must be the bits of the same
    image stored with an aligned pitch, including a resume in place."""
    h, w = 97, 131
    img = synth.make_image(h, w, seed=28, sigma=0.08)
    packed = to_gpu(img, dtype)                 # pitch 131: staged
    wide = to_gpu(img, dtype, ld=136)           # pitch 136: read through TMA directly
    a = wmc().denoise(packed, 1.0, 0.25, iters)
    b = wmc().denoise(wide, 1.0, 0.25, iters)
    assert torch.equal(a, b)
    u = wmc().denoise(packed, 1.0, 0.25, 3)
    wmc().denoise(packed, 1.0, 0.25, iters, u0=u, out=u)
    assert torch.equal(u, wmc().denoise(wide, 1.0, 0.25, 3 + iters))
