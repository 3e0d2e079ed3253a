"""wmc_denoise_noalloc: denoising for callers that cannot allocate device scratch memory.

Some callers cannot call cudaMalloc: code that runs inside another framework's memory pool,
hosts that forbid allocation once they have started, bindings that hold only existing image
pointers.  This entry point runs the same flow as wmc_denoise but takes its scratch from a fixed
array inside the library instead of a caller-provided workspace.  The file is collected last so
that a run stopping at the first failure has already run every other test; it also passes on its
own in a fresh process, where the first call performs the per-device set-up.  Every call goes
through the C ABI (ctypes) and is compared with wmc_denoise on the same input: both launch the same
kernels in the same order, so the results must agree bit for bit, on two calls in a row (the
calls share the one scratch array, which keeps the previous call's contents).
"""
import numpy as np
import pytest
import torch

from paper_1903_07189_gb300 import synth

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1903_07189_gb300 import wmc
    return wmc, wmc.load()


def _noalloc(lib, f, u, lam, step, iters, bnd=0, u0=None):
    from paper_1903_07189_gb300 import wmc
    h, w = f.shape
    return lib.wmc_denoise_noalloc(f.data_ptr(), None if u0 is None else u0.data_ptr(), u.data_ptr(), h, w,
                                   f.stride(0), wmc.DTYPES[f.dtype], lam, step, iters, bnd,
                                   torch.cuda.current_stream().cuda_stream)


def test_noalloc_matches_workspace_entry_point_twice():
    wmc, lib = _lib()
    cases = [(synth.make_image(333, 517, seed=31, sigma=0.08), 1.0, 0.25, 13, 0),
             (synth.make_image(1024, 777, seed=32, sigma=0.03), 1.7, 0.18, 9, 1)]
    for img, lam, step, iters, bnd in cases:  # two calls in a row share the one scratch array
        f = torch.from_numpy(img).cuda()
        u = torch.full_like(f, float("nan"))
        assert _noalloc(lib, f, u, lam, step, iters, bnd) == 0, lib.wmc_last_error()
        ref = wmc.denoise(f, lam, step, iters, ("replicate", "zero")[bnd])
        torch.cuda.synchronize()
        assert torch.equal(u, ref), f.shape
        assert lib.wmc_denoise_noalloc_status(torch.cuda.current_stream().cuda_stream) == 0


@pytest.mark.parametrize("iters", [5, 9])
def test_noalloc_resumes_in_place(iters):
    """u0 == u: the first launch writes the scratch image; with an odd number of 4-step launches
    (iters 9: 4 + 4 + 1) the result ends in the scratch and is copied back."""
    wmc, lib = _lib()
    f = torch.from_numpy(synth.make_image(211, 300, seed=33, sigma=0.06)).cuda()
    u = wmc.denoise(f, 1.2, 0.2, 3)
    assert _noalloc(lib, f, u, 1.2, 0.2, iters, 0, u0=u) == 0, lib.wmc_last_error()
    ref = wmc.denoise(f, 1.2, 0.2, 3 + iters)
    torch.cuda.synchronize()
    assert torch.equal(u, ref)


def test_noalloc_bf16_storage():
    wmc, lib = _lib()
    f = torch.from_numpy(synth.make_image(700, 1300, seed=34, sigma=0.05)).cuda().to(torch.bfloat16)
    for iters in (6, 11):
        u = torch.empty_like(f)
        assert _noalloc(lib, f, u, 1.0, 0.25, iters) == 0, lib.wmc_last_error()
        ref = wmc.denoise(f, 1.0, 0.25, iters)
        torch.cuda.synchronize()
        assert torch.equal(u, ref), iters


def test_noalloc_reports_a_timed_out_wait():
    """The status word at the start of the fixed scratch is made to read WMC_ERR_TIMEOUT by the
    self-test's wait that nothing completes (10 ms); wmc_denoise_noalloc_status reports it, and
    the next wmc_denoise_noalloc call clears it and still gives the exact result."""
    wmc, lib = _lib()
    st = torch.cuda.current_stream().cuda_stream
    f = torch.from_numpy(synth.make_image(150, 170, seed=35)).cuda()
    u = torch.empty_like(f)
    assert _noalloc(lib, f, u, 1.0, 0.25, 8) == 0
    assert lib.wmc_denoise_noalloc_status(st) == 0
    wmc.selftest_status_timeout("noalloc", 10_000_000)
    assert lib.wmc_denoise_noalloc_status(st) == 5  # WMC_ERR_TIMEOUT
    again = torch.empty_like(f)
    assert _noalloc(lib, f, again, 1.0, 0.25, 8) == 0
    assert lib.wmc_denoise_noalloc_status(st) == 0
    assert torch.equal(again, u)


def test_noalloc_rejects_images_beyond_its_scratch():
    wmc, lib = _lib()
    limit = lib.wmc_denoise_noalloc_max_bytes()
    assert limit == 32 << 20
    f = torch.zeros((4096, 4096), device="cuda")  # needs 64 MiB + 256 B of scratch in FP32
    u = torch.zeros_like(f)
    assert _noalloc(lib, f, u, 1.0, 0.25, 3) == 1
    assert b"scratch" in lib.wmc_last_error()
    assert torch.count_nonzero(u).item() == 0  # nothing was launched
