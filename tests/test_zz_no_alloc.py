"""wmc_denoise_noalloc: denoising for callers that cannot allocate device scratch memory.

It runs the same flow as wmc_denoise but takes its scratch from a fixed array inside the
library instead of a caller-provided workspace.  This file is collected last so that a run
stopping at the first failure has already run every other test; it also passes on its own in a
fresh process, where the first call performs the per-device set-up.  Each call goes through the
C ABI (ctypes) and is compared with wmc_denoise on the same input, within the parity tolerance
the other tests use (1e-5 of the input range), on two calls in a row.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1903_07189_gb300 import synth

pytestmark = pytest.mark.gpu
TOL_REL = 1e-5


def _lib():
    from paper_1903_07189_gb300 import wmc
    return wmc, wmc.load()


def _noalloc(lib, f, u, lam, step, iters, bnd=0):
    h, w = f.shape
    return lib.wmc_denoise_noalloc(f.data_ptr(), None, u.data_ptr(), h, w, f.stride(0), 0, lam, step,
                                   iters, bnd, torch.cuda.current_stream().cuda_stream)


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
        R = float(img.max() - img.min())
        err = (u.double() - ref.double()).abs().max().item()
        assert err <= TOL_REL * R, (err, f.shape)


def test_noalloc_rejects_images_beyond_its_scratch():
    wmc, lib = _lib()
    limit = lib.wmc_denoise_noalloc_max_bytes()
    assert limit == 32 << 20
    f = torch.zeros((4096, 4096), device="cuda")  # needs 64 MiB + 256 B of scratch in FP32
    u = torch.zeros_like(f)
    assert _noalloc(lib, f, u, 1.0, 0.25, 3) == 1
    assert b"scratch" in lib.wmc_last_error()
    assert torch.count_nonzero(u).item() == 0  # nothing was launched
