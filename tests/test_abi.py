"""The C ABI on the host: libwmc.so builds and loads, exports every function include/*.h
declares, and rejects bad arguments before touching the GPU.  No kernel is launched here:
every call below fails validation, which happens on the host."""
import ctypes
import glob
import os
import re

import pytest

from paper_1903_07189_gb300 import build, wmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

OK, INVALID, ALIAS, UNSUPPORTED, CUDA, TIMEOUT, WORKSPACE = range(7)


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(wmc_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return wmc.load()


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ["wmc_eval", "wmc_denoise", "wmc_energy", "wmc_status_string", "wmc_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(wmc.SIGNATURES)


def test_python_layer_names():
    """The user-facing calls: evaluation, denoising (single, batched), the autograd node."""
    for name in ["eval", "denoise", "denoise_batched", "energy", "WMCDenoise", "unrolled_denoise",
                 "denoise_l1", "eval_fd", "denoise_fd", "shard_lpt"]:
        assert callable(getattr(wmc, name)), name
    assert wmc.WMCDenoise is wmc.UnrolledDenoise


def test_library_is_built_for_sm_103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(build.LIB)


def test_status_strings(lib):
    assert lib.wmc_status_string(0) == b"WMC_OK"
    assert lib.wmc_status_string(2) == b"WMC_ERR_ALIAS"
    assert lib.wmc_status_string(99) == b"WMC_ERR_UNKNOWN"
    assert lib.wmc_version() >= 100


def _flag_bytes(h, w):
    """One 4-byte flag per tile of the largest tile grid of a multi-step launch: output tiles of
    (130 - 2T) x (4 NW + 2 - 2T) cells for T = 2..8 steps and NW = 16 or 8 warps, rounded up to
    256 bytes."""
    most = max(-(-w // (130 - 2 * T)) * -(-h // (4 * nw + 2 - 2 * T)) for T in range(2, 9) for nw in (16, 8))
    return -(-4 * most // 256) * 256


def test_workspace_sizes(lib):
    assert lib.wmc_denoise_workspace_size(0, 5, 5, 0) == 0
    # status word (256 bytes) + one image rounded up to 256 bytes + the tile flags
    assert _flag_bytes(3, 5) == 256 and _flag_bytes(4096, 4096) == 129 * 256  # 36 x 228 tiles
    assert lib.wmc_denoise_workspace_size(3, 5, 8, 0) == 256 + 256 + 256
    assert lib.wmc_denoise_workspace_size(100, 100, 128, 1) == 256 + (100 * 128 * 2 + 255) // 256 * 256 + 256
    assert lib.wmc_denoise_workspace_size(4096, 4096, 4096, 0) == 256 + 4096 * 4096 * 4 + 129 * 256
    assert lib.wmc_denoise_workspace_size(4, 5, 4, 0) == 0  # ld < w
    # pitches that are not a multiple of 16 bytes are staged: three images of the aligned pitch
    # (FP32: a multiple of 4 elements; 16-bit: of 8), or one of pitch ld if that is larger
    assert lib.wmc_denoise_workspace_size(10, 10, 10, 0) == 256 + 3 * 512 + 256  # pitch 12: 480 -> 512 B
    assert lib.wmc_denoise_workspace_size(10, 10, 12, 0) == 256 + 512 + 256      # aligned: one image
    assert lib.wmc_denoise_workspace_size(10, 10, 11, 1) == 256 + 3 * 512 + 256  # 16-bit, pitch 16: 320 -> 512 B
    assert lib.wmc_denoise_workspace_size(2, 3, 201, 0) == 256 + (2 * 201 * 4 + 255) // 256 * 256 + 256
    # f, U^0 and U on the device, then wmc_denoise's workspace (tile flags included)
    assert lib.wmc_denoise_host_workspace_size(10, 10, 10, 0) == 3 * 512 + 256 + 3 * 512 + 256
    assert lib.wmc_energy_workspace_size(10, 10) % 256 == 0


# Fake, never-dereferenced addresses: every call below is rejected before any launch.
A, B = 0x10000000, 0x20000000


def _err(lib):
    return lib.wmc_last_error().decode()


def test_eval_validation(lib):
    assert lib.wmc_eval(A, B, -1, 4, 4, 4, 0, 0, None) == INVALID
    assert lib.wmc_eval(A, B, 4, 4, 3, 4, 0, 0, None) == INVALID and "leading" in _err(lib)
    assert lib.wmc_eval(A, B, 4, 4, 4, 4, 7, 0, None) == INVALID and "dtype" in _err(lib)
    assert lib.wmc_eval(A, B, 4, 4, 4, 4, 0, 5, None) == INVALID and "boundary" in _err(lib)
    assert lib.wmc_eval(None, B, 4, 4, 4, 4, 0, 0, None) == INVALID
    assert lib.wmc_eval(A, A + 8, 4, 4, 4, 4, 0, 0, None) == ALIAS
    assert lib.wmc_eval(A, B, 0, 4, 4, 4, 0, 0, None) == OK  # empty: nothing enqueued


def _denoise(lib, f, u0, u, h, w, ld, dtype=0, lam=1.0, step=0.25, iters=3, bnd=0, ws=None, wsb=0):
    return lib.wmc_denoise(f, u0, u, h, w, ld, dtype, lam, step, iters, bnd, ws, wsb, None)


def test_denoise_validation(lib):
    assert _denoise(lib, A, None, B, 4, 4, 4, lam=-1.0) == INVALID and "lambda" in _err(lib)
    assert _denoise(lib, A, None, B, 4, 4, 4, lam=float("nan")) == INVALID
    assert _denoise(lib, A, None, B, 4, 4, 4, step=0.0) == INVALID and "step" in _err(lib)
    assert _denoise(lib, A, None, B, 4, 4, 4, step=float("inf")) == INVALID
    assert _denoise(lib, A, None, B, 4, 4, 4, iters=-2) == INVALID
    assert _denoise(lib, None, None, B, 4, 4, 4) == INVALID
    assert _denoise(lib, A, None, None, 4, 4, 4) == INVALID
    assert _denoise(lib, A, None, A + 4, 4, 4, 4) == ALIAS and "f" in _err(lib)
    assert _denoise(lib, A, A + 64, A + 4096, 4, 4, 4, ws=None) == WORKSPACE
    assert _denoise(lib, A, None, B, 4, 4, 4, ws=0x30000000, wsb=16) == WORKSPACE
    assert _denoise(lib, A, None, B, 4, 4, 4, ws=0x30000010, wsb=4096) == WORKSPACE and "aligned" in _err(lib)
    assert _denoise(lib, A, None, B, 4, 4, 4, ws=B, wsb=4096) == ALIAS
    assert _denoise(lib, A, None, B, 0, 0, 0) == OK


def test_denoise_config_validation(lib):
    cfg = wmc.Config(9, 0)
    assert lib.wmc_denoise_ex(A, None, B, 4, 4, 4, 0, 1.0, 0.25, 3, 0, ctypes.byref(cfg), 0x30000000, 4096,
                              None) == INVALID
    cfg = wmc.Config(2, 3)  # tile shapes are 0 (default), 1 and 2
    assert lib.wmc_denoise_ex(A, None, B, 4, 4, 4, 0, 1.0, 0.25, 3, 0, ctypes.byref(cfg), 0x30000000, 4096,
                              None) == INVALID
    cfg = wmc.Config(2, -1)
    assert lib.wmc_denoise_ex(A, None, B, 4, 4, 4, 0, 1.0, 0.25, 3, 0, ctypes.byref(cfg), 0x30000000, 4096,
                              None) == INVALID


def test_energy_validation(lib):
    assert lib.wmc_energy(A, None, None, 4, 4, 4, 0, 0, None, None, 0, None) == INVALID
    assert lib.wmc_energy(None, None, None, 4, 4, 4, 0, 0, B, 0x30000000, 1 << 20, None) == INVALID
    assert lib.wmc_energy(A, None, None, 4, 4, 4, 0, 0, B, None, 0, None) == WORKSPACE


def _images(specs):
    arr = (wmc.Image * len(specs))()
    for i, (f, u, h, w, ld, lam, st) in enumerate(specs):
        arr[i] = wmc.Image(f, u, h, w, ld, lam, st)
    return arr


def test_batch_validation(lib):
    plan = wmc.BatchPlan()
    ok = (A, B, 8, 8, 8, 1.0, 0.25)
    cfg = wmc.Config(3, 0)
    imgs = _images([ok])
    assert lib.wmc_batch_plan(imgs, -1, 0, 0, None, 0x30000000, 1 << 20, ctypes.byref(plan), None) == INVALID
    assert lib.wmc_batch_plan(_images([(A, B, 8, 8, 8, float("nan"), 0.25)]), 1, 0, 0, None, 0x30000000,
                              1 << 20, ctypes.byref(plan), None) == INVALID and "image 0" in _err(lib)
    assert lib.wmc_batch_plan(_images([ok, (A + 4096, B + 64, 8, 8, 8, 1.0, 0.25)]), 2, 0, 0, None,
                              0x30000000, 1 << 20, ctypes.byref(plan), None) == ALIAS
    assert lib.wmc_batch_plan(_images([ok, (A, B + 4096, 8, 8, 8, 1.0, 0.25)]), 2, 0, 0, None,
                              0x30000000, 16, ctypes.byref(plan), None) == WORKSPACE  # shared f is fine
    assert lib.wmc_batch_plan(imgs, 1, 0, 0, ctypes.byref(wmc.Config(9, 0)), 0x30000000, 1 << 20,
                              ctypes.byref(plan), None) == INVALID
    assert lib.wmc_batch_plan(_images([(A, B, 8, 8, 7, 1.0, 0.25)]), 1, 0, 0, None, 0x30000000, 1 << 20,
                              ctypes.byref(plan), None) == INVALID
    need = lib.wmc_batch_workspace_size(imgs, 1, 0, ctypes.byref(cfg))
    assert need > 0 and need % 256 == 0
    assert lib.wmc_batch_workspace_size(_images([(A, B, 8, 8, 7, 1.0, 0.25)]), 1, 0, None) == 0
    # the 128 x 32 tile shape needs more tiles (a longer tile table) than the 128 x 64 one
    tall = _images([(A, B, 1000, 300, 300, 1.0, 0.25)])
    assert (lib.wmc_batch_workspace_size(tall, 1, 0, ctypes.byref(wmc.Config(4, 2))) >
            lib.wmc_batch_workspace_size(tall, 1, 0, ctypes.byref(wmc.Config(4, 1))) ==
            lib.wmc_batch_workspace_size(tall, 1, 0, ctypes.byref(wmc.Config(4, 0))))
    assert lib.wmc_batch_workspace_size(imgs, 1, 0, ctypes.byref(wmc.Config(4, 3))) == 0
    assert lib.wmc_batch_plan(imgs, 1, 0, 0, ctypes.byref(wmc.Config(4, 3)), 0x30000000, 1 << 20,
                              ctypes.byref(plan), None) == INVALID
    assert lib.wmc_batch_run(ctypes.byref(wmc.BatchPlan()), 5, None) == INVALID  # not planned


def test_unrolled_validation(lib):
    f = ctypes.c_void_p(0x100000)
    lam = ctypes.c_void_p(0x200000)
    u = ctypes.c_void_p(0x300000)
    ws = ctypes.c_void_p(0x10000000)
    big = 1 << 40
    assert lib.wmc_unrolled_workspace_size(0, 8, 8, 8, 4, 2) == 0
    assert lib.wmc_unrolled_workspace_size(1, 8, 8, 4, 4, 2) == 0
    assert lib.wmc_unrolled_workspace_size(1, 8, 8, 8, 4, 0) == 0
    assert lib.wmc_unrolled_workspace_size(2, 8, 8, 8, 9, 3) > lib.wmc_unrolled_workspace_size(2, 8, 8, 8, 3, 3)
    fwd = lambda *a: lib.wmc_unrolled_forward(*a)
    # n, K, ckpt_every, step, NULL pointers
    assert fwd(f, lam, 0.25, 4, 2, 0, 8, 8, 8, 0, u, ws, big, None) == INVALID
    assert fwd(f, lam, 0.25, -1, 2, 1, 8, 8, 8, 0, u, ws, big, None) == INVALID
    assert fwd(f, lam, 0.25, 4, 0, 1, 8, 8, 8, 0, u, ws, big, None) == INVALID
    assert fwd(f, lam, 0.0, 4, 2, 1, 8, 8, 8, 0, u, ws, big, None) == INVALID
    assert fwd(f, lam, float("nan"), 4, 2, 1, 8, 8, 8, 0, u, ws, big, None) == INVALID
    assert fwd(None, lam, 0.25, 4, 2, 1, 8, 8, 8, 0, u, ws, big, None) == INVALID
    assert fwd(f, None, 0.25, 4, 2, 1, 8, 8, 8, 0, u, ws, big, None) == INVALID
    assert fwd(f, lam, 0.25, 4, 2, 1, 8, 8, 8, 7, u, ws, big, None) == INVALID  # boundary
    assert fwd(f, lam, 0.25, 4, 2, 1, 8, 8, 8, 0, f, ws, big, None) == ALIAS
    assert fwd(f, lam, 0.25, 4, 2, 1, 8, 8, 8, 0, u, ws, 16, None) == WORKSPACE
    assert fwd(f, lam, 0.25, 4, 2, 1, 8, 8, 8, 0, u, ctypes.c_void_p(0x10000010), big, None) == WORKSPACE
    bwd = lib.wmc_unrolled_backward
    assert bwd(f, lam, 0.25, 4, 2, 1, 8, 8, 8, 0, u, None, lam, ws, big, None) == INVALID
    assert bwd(f, lam, 0.25, 4, 2, 1, 8, 8, 8, 0, u, u, lam, ws, big, None) == ALIAS
    assert bwd(f, lam, 0.25, 4, 2, 1, 8, 8, 8, 0, u, ctypes.c_void_p(0x400000), lam, ws, 16, None) == WORKSPACE


def test_energy_grad_validation(lib):
    u = ctypes.c_void_p(0x100000)
    g = ctypes.c_void_p(0x300000)
    assert lib.wmc_energy_grad(u, g, 8, 8, 4, 0, None) == INVALID
    assert lib.wmc_energy_grad(u, u, 8, 8, 8, 0, None) == ALIAS
    assert lib.wmc_energy_grad(u, ctypes.c_void_p(0x100010), 8, 8, 8, 0, None) == ALIAS
    assert lib.wmc_energy_grad(None, g, 8, 8, 8, 0, None) == INVALID
    assert lib.wmc_energy_grad(u, g, 8, 8, 8, 5, None) == INVALID


def test_selftest_wait_validation(lib):
    ws = ctypes.c_void_p(0x100000)
    assert lib.wmc_selftest_wait_timeout(None, 1000, None) == INVALID
    assert lib.wmc_selftest_wait_timeout(ctypes.c_void_p(0x100004), 1000, None) == WORKSPACE
    assert lib.wmc_selftest_wait_timeout(ws, 0, None) == INVALID
    assert lib.wmc_selftest_wait_timeout(ws, 2_000_000_000, None) == INVALID


def test_selftest_flag_validation(lib):
    f, u, ws = ctypes.c_void_p(0x100000), ctypes.c_void_p(0x200000), ctypes.c_void_p(0x10000000)
    need = lib.wmc_denoise_workspace_size(8, 8, 8, 0)
    assert lib.wmc_selftest_flag_timeout(None, u, 8, 8, 8, ws, need, None) == INVALID
    assert lib.wmc_selftest_flag_timeout(f, None, 8, 8, 8, ws, need, None) == INVALID
    assert lib.wmc_selftest_flag_timeout(f, u, 0, 8, 8, ws, need, None) == INVALID
    assert lib.wmc_selftest_flag_timeout(f, u, 8, 8, 4, ws, need, None) == INVALID  # ld < w
    assert lib.wmc_selftest_flag_timeout(f, f, 8, 8, 8, ws, need, None) == ALIAS
    assert lib.wmc_selftest_flag_timeout(f, u, 8, 8, 8, ws, need - 1, None) == WORKSPACE
    assert lib.wmc_selftest_flag_timeout(f, u, 8, 8, 8, ctypes.c_void_p(0x10000004), need, None) == WORKSPACE
    assert lib.wmc_selftest_flag_timeout(f, u, 8, 8, 8, ctypes.c_void_p(0x100000), 1 << 20, None) == ALIAS


def test_selftest_status_validation(lib):
    assert lib.wmc_selftest_status_timeout(0, 0, None) == INVALID
    assert lib.wmc_selftest_status_timeout(1, 2_000_000_000, None) == INVALID
    assert lib.wmc_selftest_status_timeout(2, 1000, None) == INVALID  # unknown target
    assert lib.wmc_selftest_status_timeout(-1, 1000, None) == INVALID


def test_backward_validation(lib):
    f = ctypes.c_void_p(0x100000)
    lam = ctypes.c_void_p(0x200000)
    g = ctypes.c_void_p(0x300000)
    gf = ctypes.c_void_p(0x400000)
    ws = ctypes.c_void_p(0x10000000)
    big = 1 << 40
    need = lib.wmc_backward_workspace_size(2, 8, 8, 8, 9, 3)
    assert need > lib.wmc_unrolled_workspace_size(2, 8, 8, 8, 9, 3) and need % 256 == 0
    assert lib.wmc_backward_workspace_size(0, 8, 8, 8, 9, 3) == 0
    bwd = lib.wmc_backward
    assert bwd(f, lam, 0.25, 4, 0, 1, 8, 8, 8, 0, g, gf, lam, ws, big, None) == INVALID  # ckpt_every
    assert bwd(f, lam, 0.0, 4, 2, 1, 8, 8, 8, 0, g, gf, lam, ws, big, None) == INVALID  # step
    assert bwd(None, lam, 0.25, 4, 2, 1, 8, 8, 8, 0, g, gf, lam, ws, big, None) == INVALID
    assert bwd(f, lam, 0.25, 4, 2, 1, 8, 8, 8, 0, g, gf, lam, ws, 16, None) == WORKSPACE
    assert bwd(f, lam, 0.25, 4, 2, 1, 8, 8, 8, 0, g, gf, lam, ctypes.c_void_p(0x10000010), big, None) == WORKSPACE
    assert bwd(f, lam, 0.25, 4, 2, 1, 8, 8, 8, 0, g, gf, lam, ctypes.c_void_p(0x100000 - 256), big, None) == ALIAS


def test_l1_validation(lib):
    f = ctypes.c_void_p(0x100000)
    u = ctypes.c_void_p(0x300000)
    d = ctypes.c_void_p(0x500000)
    ws = ctypes.c_void_p(0x10000000)
    need = lib.wmc_denoise_l1_workspace_size(8, 8, 8)
    assert need >= 2 * 8 * 8 * 4
    assert lib.wmc_denoise_l1_workspace_size(8, 8, 4) == 0
    call = lambda f_, u0, u_, d_, lam, step, alpha, iters, ws_=ws, nbytes=need: lib.wmc_denoise_l1(
        f_, u0, u_, d_, 8, 8, 8, lam, step, alpha, iters, 0, ws_, nbytes, None)
    assert call(f, None, u, d, -1.0, 0.1, 0.1, 3) == INVALID
    assert call(f, None, u, d, 1.0, 0.0, 0.1, 3) == INVALID
    assert call(f, None, u, d, 1.0, 0.1, 0.0, 3) == INVALID
    assert call(f, None, u, d, 1.0, 0.1, float("inf"), 3) == INVALID
    assert call(f, None, u, d, 1.0, 0.1, 0.1, -1) == INVALID
    assert call(None, None, u, d, 1.0, 0.1, 0.1, 3) == INVALID
    assert call(f, None, f, d, 1.0, 0.1, 0.1, 3) == ALIAS
    assert call(f, None, u, u, 1.0, 0.1, 0.1, 3) == ALIAS
    assert call(f, None, u, d, 1.0, 0.1, 0.1, 3, nbytes=need - 1) == WORKSPACE
    assert call(f, None, u, d, 1.0, 0.1, 0.1, 3, ws_=ctypes.c_void_p(0x10000008)) == WORKSPACE
    assert call(f, None, u, d, 1.0, 0.1, 0.1, 3, ws_=ctypes.c_void_p(0x300000)) == ALIAS


def test_batch_autotune_validation(lib):
    imgs = (wmc.Image * 1)()
    imgs[0] = wmc.Image(0x100000, 0x300000, 8, 8, 8, 1.0, 0.25)
    need = lib.wmc_batch_autotune_workspace_size(imgs, 1, 0)
    assert need > 0
    best = wmc.Config(0, 0)
    ws = ctypes.c_void_p(0x10000000)
    bad = (ctypes.c_int32 * 2)(2, 9)
    assert lib.wmc_batch_autotune(imgs, 1, 0, 0, bad, 2, 8, ws, need, ctypes.byref(best), None, None) == INVALID
    good = (ctypes.c_int32 * 1)(4)
    assert lib.wmc_batch_autotune(imgs, 1, 0, 0, good, 0, 8, ws, need, ctypes.byref(best), None, None) == INVALID
    assert lib.wmc_batch_autotune(imgs, 1, 0, 0, good, 1, 0, ws, need, ctypes.byref(best), None, None) == INVALID
    assert lib.wmc_batch_autotune(imgs, 1, 0, 0, good, 1, 8, ws, need, None, None, None) == INVALID
    cfgs = (wmc.Config * 2)(wmc.Config(4, 1), wmc.Config(4, 3))
    tune = lib.wmc_batch_autotune_configs
    assert tune(imgs, 1, 0, 0, cfgs, 2, 8, ws, need, ctypes.byref(best), None, None) == INVALID  # tile 3
    cfgs = (wmc.Config * 1)(wmc.Config(0, 1))
    assert tune(imgs, 1, 0, 0, cfgs, 1, 8, ws, need, ctypes.byref(best), None, None) == INVALID  # 0 steps
    cfgs = (wmc.Config * 1)(wmc.Config(4, 2))
    assert tune(imgs, 1, 0, 0, cfgs, 0, 8, ws, need, ctypes.byref(best), None, None) == INVALID
    assert tune(imgs, 1, 0, 0, cfgs, 1, 0, ws, need, ctypes.byref(best), None, None) == INVALID
    assert tune(imgs, 1, 0, 0, cfgs, 1, 8, ws, need, None, None, None) == INVALID


def test_unrolled_backward_workspace_alias(lib):
    f = ctypes.c_void_p(0x100000)
    lam = ctypes.c_void_p(0x200000)
    gu = ctypes.c_void_p(0x300000)
    gf = ctypes.c_void_p(0x400000)
    need = lib.wmc_unrolled_workspace_size(1, 8, 8, 8, 4, 2)
    # a workspace starting inside grad_u
    assert lib.wmc_unrolled_backward(f, lam, 0.25, 4, 2, 1, 8, 8, 8, 0, gu, gf, lam, ctypes.c_void_p(0x300000),
                                     need, None) == ALIAS
