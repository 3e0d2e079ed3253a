"""Python binding of libwmc.so (include/wmc.h): argument marshalling only.

Every entry point here hands device pointers of torch tensors, sizes and the current CUDA
stream to the C ABI; all stencil work runs in the library's CUDA kernels.  There is no CPU
fallback: if libwmc.so cannot be loaded, or a call fails, a ``WMCError`` is raised.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

DTYPES = {torch.float32: 0, torch.bfloat16: 1, torch.float16: 2}
BOUNDARY = {"replicate": 0, "zero": 1}
WORKSPACE_ALIGN = 256


class WMCError(RuntimeError):
    def __init__(self, status: int, func: str, detail: str):
        self.status = status
        super().__init__(f"{func} failed: {_STATUS.get(status, status)}: {detail}")


_STATUS = {0: "WMC_OK", 1: "WMC_ERR_INVALID_ARG", 2: "WMC_ERR_ALIAS", 3: "WMC_ERR_UNSUPPORTED",
           4: "WMC_ERR_CUDA", 5: "WMC_ERR_TIMEOUT", 6: "WMC_ERR_WORKSPACE"}


class Config(ctypes.Structure):
    _fields_ = [("steps_per_launch", ctypes.c_int32), ("tile", ctypes.c_int32)]


class Image(ctypes.Structure):
    """wmc_image_t"""
    _fields_ = [("f", ctypes.c_void_p), ("u", ctypes.c_void_p), ("h", ctypes.c_int32), ("w", ctypes.c_int32),
                ("ld", ctypes.c_int64), ("lam", ctypes.c_float), ("step", ctypes.c_float)]


class BatchPlan(ctypes.Structure):
    """wmc_batch_t (opaque, caller-owned)"""
    _fields_ = [("opaque", ctypes.c_int64 * 16)]


_lib = None

# name -> (restype, argtypes) for every symbol declared in include/wmc.h
_vp, _i32, _i64, _f32, _sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
SIGNATURES = {
    "wmc_eval": (_i32, [_vp, _vp, _i32, _i32, _i64, _i64, _i32, _i32, _vp]),
    "wmc_denoise_workspace_size": (_sz, [_i32, _i32, _i64, _i32]),
    "wmc_eval_fd": (_i32, [_vp, _vp, _i32, _i32, _i64, _i64, _i32, _i32, _vp]),
    "wmc_denoise_fd": (_i32, [_vp, _vp, _vp, _i32, _i32, _i64, _i32, _f32, _f32, _i32, _i32, _vp, _sz, _vp]),
    "wmc_denoise": (_i32, [_vp, _vp, _vp, _i32, _i32, _i64, _i32, _f32, _f32, _i32, _i32, _vp, _sz, _vp]),
    "wmc_denoise_ex": (_i32, [_vp, _vp, _vp, _i32, _i32, _i64, _i32, _f32, _f32, _i32, _i32,
                              ctypes.POINTER(Config), _vp, _sz, _vp]),
    "wmc_denoise_status": (_i32, [_vp, _vp]),
    "wmc_denoise_noalloc_max_bytes": (_sz, []),
    "wmc_denoise_cluster_size": (_i32, [_i32, _i32, _i32]),
    "wmc_denoise_noalloc": (_i32, [_vp, _vp, _vp, _i32, _i32, _i64, _i32, _f32, _f32, _i32, _i32, _vp]),
    "wmc_denoise_noalloc_status": (_i32, [_vp]),
    "wmc_selftest_status_timeout": (_i32, [_i32, _i64, _vp]),
    "wmc_denoise_host_workspace_size": (_sz, [_i32, _i32, _i64, _i32]),
    "wmc_denoise_host": (_i32, [_vp, _vp, _vp, _i32, _i32, _i64, _i32, _f32, _f32, _i32, _i32, _vp, _sz,
                                _vp]),
    "wmc_energy_workspace_size": (_sz, [_i32, _i32]),
    "wmc_energy": (_i32, [_vp, _vp, _vp, _i32, _i32, _i64, _i32, _i32, _vp, _vp, _sz, _vp]),
    "wmc_batch_workspace_size": (_sz, [ctypes.POINTER(Image), _i32, _i32, ctypes.POINTER(Config)]),
    "wmc_batch_plan": (_i32, [ctypes.POINTER(Image), _i32, _i32, _i32, ctypes.POINTER(Config), _vp, _sz,
                              ctypes.POINTER(BatchPlan), _vp]),
    "wmc_batch_run": (_i32, [ctypes.POINTER(BatchPlan), _i32, _vp]),
    "wmc_denoise_batched": (_i32, [ctypes.POINTER(Image), _i32, _i32, _i32, _i32, _vp, _sz, _vp]),
    "wmc_batch_autotune_workspace_size": (_sz, [ctypes.POINTER(Image), _i32, _i32]),
    "wmc_batch_autotune": (_i32, [ctypes.POINTER(Image), _i32, _i32, _i32, ctypes.POINTER(ctypes.c_int32), _i32,
                                  _i32, _vp, _sz, ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_float), _vp]),
    "wmc_batch_autotune_configs": (_i32, [ctypes.POINTER(Image), _i32, _i32, _i32, ctypes.POINTER(Config), _i32,
                                          _i32, _vp, _sz, ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_float),
                                          _vp]),
    "wmc_denoise_l1_workspace_size": (_sz, [_i32, _i32, _i64]),
    "wmc_denoise_l1": (_i32, [_vp, _vp, _vp, _vp, _i32, _i32, _i64, _f32, _f32, _f32, _i32, _i32, _vp, _sz,
                              _vp]),
    "wmc_unrolled_workspace_size": (_sz, [_i32, _i32, _i32, _i64, _i32, _i32]),
    "wmc_unrolled_forward": (_i32, [_vp, _vp, _f32, _i32, _i32, _i32, _i32, _i32, _i64, _i32, _vp, _vp, _sz,
                                    _vp]),
    "wmc_unrolled_backward": (_i32, [_vp, _vp, _f32, _i32, _i32, _i32, _i32, _i32, _i64, _i32, _vp, _vp, _vp,
                                     _vp, _sz, _vp]),
    "wmc_backward_workspace_size": (_sz, [_i32, _i32, _i32, _i64, _i32, _i32]),
    "wmc_backward": (_i32, [_vp, _vp, _f32, _i32, _i32, _i32, _i32, _i32, _i64, _i32, _vp, _vp, _vp, _vp, _sz,
                            _vp]),
    "wmc_energy_grad": (_i32, [_vp, _vp, _i32, _i32, _i64, _i32, _vp]),
    "wmc_shard_lpt": (_i32, [_vp, _i32, _i32, _vp, _vp]),
    "wmc_selftest_wait_timeout": (_i32, [_vp, _i64, _vp]),
    "wmc_selftest_flag_timeout": (_i32, [_vp, _vp, _i32, _i32, _i64, _vp, _sz, _vp]),
    "wmc_eval_status": (_i32, [_vp]),
    "wmc_probe_fma_threads": (_i32, []),
    "wmc_probe_fma": (_i32, [_vp, _i32, _i32, _vp]),
    "wmc_status_string": (ctypes.c_char_p, [_i32]),
    "wmc_last_error": (ctypes.c_char_p, []),
    "wmc_version": (_i32, []),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libwmc.so (building it first if needed); raises if that is impossible."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise WMCError(3, "load", f"{path} not found; run build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status: int, func: str):
    if status != 0:
        raise WMCError(status, func, load().wmc_last_error().decode())


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _img(t: torch.Tensor, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dim() != 2:
        raise ValueError(f"{name} must be 2-D (H, W)")
    if t.dtype not in DTYPES:
        raise ValueError(f"{name}: unsupported dtype {t.dtype}")
    if t.stride(1) != 1 or (t.size(0) > 1 and t.stride(0) < t.size(1)):
        raise ValueError(f"{name} must be row-major with unit column stride")
    return t.data_ptr(), t.size(0), t.size(1), max(t.stride(0), t.size(1))


def _workspace(nbytes: int, device) -> torch.Tensor:
    # torch's caching allocator hands out 512-byte aligned blocks, above WORKSPACE_ALIGN.
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)


def eval(u: torch.Tensor, boundary: str = "replicate", out: torch.Tensor | None = None) -> torch.Tensor:
    """H^w(U) (Sec. IV-B: Eq. conv + Eq. act) of a 2-D CUDA tensor."""
    p, h, w, ld = _img(u, "u")
    if out is None:
        out = torch.empty_like(u, memory_format=torch.contiguous_format)
    po, ho, wo, ldo = _img(out, "out")
    if (ho, wo) != (h, w) or out.dtype != u.dtype:
        raise ValueError("out must match u in shape and dtype")
    _check(load().wmc_eval(p, po, h, w, ld, ldo, DTYPES[u.dtype], BOUNDARY[boundary], _stream(u.device)),
           "wmc_eval")
    return out


def eval_status(device=None):
    """Raise WMCError(WMC_ERR_TIMEOUT) if a bounded device wait of an evaluation since the last
    check gave up (synchronises the current stream; clears the word)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    _check(load().wmc_eval_status(_stream(dev)), "wmc_eval_status")


def eval_fd(u: torch.Tensor, boundary: str = "replicate", out: torch.Tensor | None = None) -> torch.Tensor:
    """Conventional finite-difference WMC of Eq. rhs (the comparator of Sec. V-D)."""
    p, h, w, ld = _img(u, "u")
    if out is None:
        out = torch.empty_like(u, memory_format=torch.contiguous_format)
    po, ho, wo, ldo = _img(out, "out")
    if (ho, wo) != (h, w) or out.dtype != u.dtype:
        raise ValueError("out must match u in shape and dtype")
    _check(load().wmc_eval_fd(p, po, h, w, ld, ldo, DTYPES[u.dtype], BOUNDARY[boundary], _stream(u.device)),
           "wmc_eval_fd")
    return out


def denoise_fd(f: torch.Tensor | None, lam: float = 1.0, step: float = 0.1, iters: int = 100,
               boundary: str = "replicate", u0: torch.Tensor | None = None, out: torch.Tensor | None = None,
               workspace: torch.Tensor | None = None) -> torch.Tensor:
    """The flow of `denoise` with the finite-difference H of Eq. rhs (f None: mean-curvature flow
    from u0)."""
    ref = f if f is not None else u0
    if ref is None:
        raise ValueError("f or u0 is required")
    p, h, w, ld = _img(ref, "f" if f is not None else "u0")
    if out is None:
        out = torch.empty_strided(ref.shape, ref.stride(), dtype=ref.dtype, device=ref.device)
    for t, n in [(f, "f"), (u0, "u0"), (out, "out")]:
        if t is not None:
            _, h2, w2, ld2 = _img(t, n)
            if (h2, w2, ld2) != (h, w, ld) or t.dtype != ref.dtype:
                raise ValueError(f"{n} must match in shape, pitch and dtype")
    lib = load()
    if workspace is None:
        workspace = _workspace(lib.wmc_denoise_workspace_size(h, w, ld, DTYPES[ref.dtype]), ref.device)
    _check(lib.wmc_denoise_fd(f.data_ptr() if f is not None else None, u0.data_ptr() if u0 is not None else None,
                              out.data_ptr(), h, w, ld, DTYPES[ref.dtype], float(lam), float(step), int(iters),
                              BOUNDARY[boundary], workspace.data_ptr(), workspace.numel(), _stream(ref.device)),
           "wmc_denoise_fd")
    return out


def default_step(lam: float) -> float:
    """0.5 / (1 + lambda): half the largest step that keeps the max principle."""
    return 0.5 / (1.0 + lam)


def denoise(f: torch.Tensor | None, lam: float = 1.0, step: float | None = None, iters: int = 100,
            boundary: str = "replicate", u0: torch.Tensor | None = None, out: torch.Tensor | None = None,
            steps_per_launch: int = 0, workspace: torch.Tensor | None = None, tile: int = 0) -> torch.Tensor:
    """`iters` Jacobi steps of U <- U + step*(lam*H^w(U) - (U - f)) (Sec. V-B, A = I).

    f = None gives the mean-curvature flow U <- U + step*lam*H^w(U) (Eq. MCF) from u0.
    steps_per_launch and tile pick the kernel configuration (0: defaults; tile 1: 128 x 64
    regions, 2: 128 x 32); the result does not depend on them.
    """
    ref = f if f is not None else u0
    if ref is None:
        raise ValueError("need f or u0")
    if step is None:
        step = default_step(lam if f is not None else 0.0)
    pr, h, w, ld = _img(ref, "f" if f is not None else "u0")
    pf = _img(f, "f")[0] if f is not None else None
    pu0 = None
    if u0 is not None:
        pu0, h2, w2, ld2 = _img(u0, "u0")
        if (h2, w2, ld2) != (h, w, ld) or u0.dtype != ref.dtype:
            raise ValueError("u0 must match f in shape, pitch and dtype")
    if out is None:
        out = torch.empty_strided(ref.shape, ref.stride(), dtype=ref.dtype, device=ref.device)
    po, ho, wo, ldo = _img(out, "out")
    if (ho, wo, ldo) != (h, w, ld) or out.dtype != ref.dtype:
        raise ValueError("out must match f in shape, pitch and dtype")
    lib = load()
    dt = DTYPES[ref.dtype]
    need = lib.wmc_denoise_workspace_size(h, w, ld, dt)
    if workspace is None:
        workspace = _workspace(need, ref.device)
    cfg = Config(int(steps_per_launch), int(tile))
    _check(lib.wmc_denoise_ex(pf, pu0, po, h, w, ld, dt, float(lam), float(step), int(iters),
                              BOUNDARY[boundary], ctypes.byref(cfg), workspace.data_ptr(),
                              workspace.numel(), _stream(ref.device)), "wmc_denoise")
    return out


def cluster_size(h: int, w: int, iters: int, device=None) -> int:
    """CTAs of the one-launch cluster path that the default configuration takes for an h x w
    image and `iters` iterations on `device` (0: the multi-launch path)."""
    lib = load()
    with torch.cuda.device(device if device is not None else torch.cuda.current_device()):
        return int(lib.wmc_denoise_cluster_size(int(h), int(w), int(iters)))


def mcf(u0: torch.Tensor, step: float = 0.25, iters: int = 100, boundary: str = "replicate", **kw):
    """Mean-curvature flow U <- U + step*H^w(U) (Eq. MCF)."""
    return denoise(None, lam=1.0, step=step, iters=iters, boundary=boundary, u0=u0, **kw)


def denoise_host(f: torch.Tensor, lam: float = 1.0, step: float | None = None, iters: int = 100,
                 boundary: str = "replicate", out: torch.Tensor | None = None,
                 workspace: torch.Tensor | None = None, device="cuda", stream=None) -> torch.Tensor:
    """wmc_denoise_host: f and the result live in (preferably pinned) HOST memory; the library
    copies in, runs the flow and copies out on `stream`.  Returns after enqueueing; the caller
    synchronises the stream before reading `out`."""
    if f.is_cuda or f.dim() != 2 or f.dtype not in DTYPES or not f.is_contiguous():
        raise ValueError("f must be a contiguous 2-D host tensor")
    h, w = f.shape
    if out is None:
        out = torch.empty_like(f, pin_memory=f.is_pinned())
    if step is None:
        step = default_step(lam)
    lib = load()
    dt = DTYPES[f.dtype]
    need = lib.wmc_denoise_host_workspace_size(h, w, w, dt)
    if workspace is None:
        workspace = _workspace(need, device)
    st = stream.cuda_stream if stream is not None else _stream(torch.device(device))
    _check(lib.wmc_denoise_host(f.data_ptr(), None, out.data_ptr(), h, w, w, dt, float(lam), float(step),
                                int(iters), BOUNDARY[boundary], workspace.data_ptr(), workspace.numel(), st),
           "wmc_denoise_host")
    return out


def check_status(workspace: torch.Tensor):
    """Raise WMCError(WMC_ERR_TIMEOUT) if a bounded device wait in the last flow call that used
    `workspace` gave up (synchronises the current stream)."""
    _check(load().wmc_denoise_status(workspace.data_ptr(), _stream(workspace.device)), "wmc_denoise_status")


def selftest_wait_timeout(workspace: torch.Tensor, limit_ns: int = 10_000_000):
    """Make one bounded device wait run out on purpose (wmc_selftest_wait_timeout): afterwards
    check_status(workspace) raises WMCError(WMC_ERR_TIMEOUT)."""
    _check(load().wmc_selftest_wait_timeout(workspace.data_ptr(), int(limit_ns), _stream(workspace.device)),
           "wmc_selftest_wait_timeout")


SELFTEST_TARGETS = {"eval": 0, "noalloc": 1}


def selftest_flag_timeout(f: torch.Tensor, out: torch.Tensor, workspace: torch.Tensor):
    """Make the per-tile flag wait of a chained flow launch run out on purpose
    (wmc_selftest_flag_timeout): out gets 4 flow steps from f, and check_status(workspace) then
    raises WMC_ERR_TIMEOUT until the next flow call on that workspace."""
    p, h, w, ld = _img(f, "f")
    po, ho, wo, ldo = _img(out, "out")
    if (ho, wo, ldo) != (h, w, ld) or f.dtype != torch.float32 or out.dtype != torch.float32:
        raise ValueError("f and out must be FP32 images of one shape and pitch")
    _check(load().wmc_selftest_flag_timeout(p, po, h, w, ld, workspace.data_ptr(), workspace.numel(),
                                            _stream(f.device)), "wmc_selftest_flag_timeout")
    return out


def selftest_status_timeout(target: str, limit_ns: int = 10_000_000, device=None):
    """Make one bounded device wait run out on purpose against a status word the library holds
    per device ("eval": the word eval_status reads; "noalloc": the word at the start of the fixed
    scratch of wmc_denoise_noalloc)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    _check(load().wmc_selftest_status_timeout(SELFTEST_TARGETS[target], int(limit_ns), _stream(dev)),
           "wmc_selftest_status_timeout")


def denoise_host_workspace_size(h: int, w: int, dtype=torch.float32) -> int:
    return load().wmc_denoise_host_workspace_size(h, w, w, DTYPES[dtype])


def energy(u: torch.Tensor, f: torch.Tensor | None = None, clean: torch.Tensor | None = None,
           boundary: str = "replicate", out: torch.Tensor | None = None,
           workspace: torch.Tensor | None = None) -> torch.Tensor:
    """(sum|H^w|, 1/2 sum (U-f)^2, sum (U-clean)^2) as a float64 CUDA tensor of 3 values."""
    p, h, w, ld = _img(u, "u")
    for t, n in [(f, "f"), (clean, "clean")]:
        if t is not None:
            _, h2, w2, ld2 = _img(t, n)
            if (h2, w2, ld2) != (h, w, ld) or t.dtype != u.dtype:
                raise ValueError(f"{n} must match u in shape, pitch and dtype")
    lib = load()
    if out is None:
        out = torch.empty(3, dtype=torch.float64, device=u.device)
    if workspace is None:
        workspace = _workspace(lib.wmc_energy_workspace_size(h, w), u.device)
    _check(lib.wmc_energy(p, f.data_ptr() if f is not None else None,
                          clean.data_ptr() if clean is not None else None, h, w, ld, DTYPES[u.dtype],
                          BOUNDARY[boundary], out.data_ptr(), workspace.data_ptr(), workspace.numel(),
                          _stream(u.device)), "wmc_energy")
    return out


class Batch:
    """A planned batch of images of any sizes, each with its own lambda and step (wmc_batch_plan).

    fs: 2-D CUDA tensors of one dtype (U^0 = f); outs: optional output tensors (same shapes and
    pitches).  run(iters) enqueues wmc_batch_run on the current stream: kernel launches only, so
    it can be captured into a CUDA graph.  The plan keeps references to fs, outs and its
    workspace, which must outlive every run.
    """

    def __init__(self, fs, lams, steps=None, outs=None, boundary: str = "replicate",
                 steps_per_launch: int = 0, tile: int = 0):
        if not fs:
            raise ValueError("empty batch")
        dt = fs[0].dtype
        if steps is None:
            steps = [default_step(l) for l in lams]
        if outs is None:
            outs = [torch.empty_strided(f.shape, f.stride(), dtype=f.dtype, device=f.device) for f in fs]
        if not (len(fs) == len(lams) == len(steps) == len(outs)):
            raise ValueError("fs, lams, steps and outs must have the same length")
        n = len(fs)
        imgs = (Image * n)()
        for i, (f, u, l, st) in enumerate(zip(fs, outs, lams, steps)):
            pf, h, w, ld = _img(f, f"fs[{i}]")
            pu, h2, w2, ld2 = _img(u, f"outs[{i}]")
            if (h2, w2, ld2) != (h, w, ld) or f.dtype != dt or u.dtype != dt:
                raise ValueError(f"image {i}: f and out must share shape, pitch and dtype")
            imgs[i] = Image(pf, pu, h, w, ld, float(l), float(st))
        lib = load()
        self.cfg = Config(int(steps_per_launch), int(tile))
        self.dtype = DTYPES[dt]
        size = lib.wmc_batch_workspace_size(imgs, n, self.dtype, ctypes.byref(self.cfg))
        if size == 0:
            raise WMCError(1, "wmc_batch_workspace_size", "invalid batch")
        self.device = fs[0].device
        self.workspace = _workspace(size, self.device)
        self.plan = BatchPlan()
        _check(lib.wmc_batch_plan(imgs, n, self.dtype, BOUNDARY[boundary], ctypes.byref(self.cfg),
                                  self.workspace.data_ptr(), self.workspace.numel(), ctypes.byref(self.plan),
                                  _stream(self.device)), "wmc_batch_plan")
        self.fs, self.outs, self.imgs, self.n = list(fs), outs, imgs, n

    def run(self, iters: int):
        _check(load().wmc_batch_run(ctypes.byref(self.plan), int(iters), _stream(self.device)), "wmc_batch_run")
        return self.outs

    def check_status(self):
        check_status(self.workspace)


def batch_autotune(fs, lams, steps=None, outs=None, boundary: str = "replicate", candidates=None,
                   trial_iters: int = 24):
    """Time the batch at each candidate configuration (wmc_batch_autotune_configs): candidates are
    (steps_per_launch, tile) pairs, None = both tile shapes x steps {2, 3, 4, 5, 6, 8}.  Returns
    ((best steps per launch, best tile), {(steps, tile): ms per iteration}).  Writes the outputs."""
    if not fs:
        raise ValueError("empty batch")
    dt = fs[0].dtype
    if steps is None:
        steps = [default_step(l) for l in lams]
    if outs is None:
        outs = [torch.empty_strided(f.shape, f.stride(), dtype=f.dtype, device=f.device) for f in fs]
    n = len(fs)
    imgs = (Image * n)()
    for i, (f, u, l, st) in enumerate(zip(fs, outs, lams, steps)):
        pf, h, w, ld = _img(f, f"fs[{i}]")
        pu, h2, w2, ld2 = _img(u, f"outs[{i}]")
        if (h2, w2, ld2) != (h, w, ld) or f.dtype != dt or u.dtype != dt:
            raise ValueError(f"image {i}: f and out must share shape, pitch and dtype")
        imgs[i] = Image(pf, pu, h, w, ld, float(l), float(st))
    lib = load()
    size = lib.wmc_batch_autotune_workspace_size(imgs, n, DTYPES[dt])
    if size == 0:
        raise WMCError(1, "wmc_batch_autotune_workspace_size", "invalid batch")
    ws = _workspace(size, fs[0].device)
    if candidates is None:
        candidates = [(T, tile) for tile in (1, 2) for T in (2, 3, 4, 5, 6, 8)]
    cand = (Config * len(candidates))(*[Config(int(T), int(tile)) for T, tile in candidates])
    times = (ctypes.c_float * len(candidates))()
    best = Config(0, 0)
    _check(lib.wmc_batch_autotune_configs(imgs, n, DTYPES[dt], BOUNDARY[boundary], cand, len(candidates),
                                          int(trial_iters), ws.data_ptr(), ws.numel(), ctypes.byref(best), times,
                                          _stream(fs[0].device)), "wmc_batch_autotune_configs")
    return (best.steps_per_launch, best.tile), {tuple(c): float(t) for c, t in zip(candidates, times)}


def denoise_batched(fs, lams, steps=None, iters: int = 100, boundary: str = "replicate", outs=None,
                    steps_per_launch: int = 0, tile: int = 0):
    """Plan and run one batch; returns the output tensors."""
    return Batch(fs, lams, steps, outs, boundary, steps_per_launch, tile).run(iters)


def denoise_l1(f: torch.Tensor, lam: float = 1.0, step: float = 0.1, alpha: float = 0.1,
               iters: int = 100, boundary: str = "replicate", u0: torch.Tensor | None = None,
               d: torch.Tensor | None = None, out: torch.Tensor | None = None,
               workspace: torch.Tensor | None = None) -> torch.Tensor:
    """L1-fidelity primal-dual iteration (Sec. V-C, A = I) on an FP32 CUDA image.  d, if given,
    holds d^0 and receives d^iters (None: d^0 = 0)."""
    p, h, w, ld = _img(f, "f")
    if f.dtype != torch.float32:
        raise ValueError("denoise_l1 supports float32 only")
    if out is None:
        out = torch.empty_strided(f.shape, f.stride(), dtype=f.dtype, device=f.device)
    for t, n in [(u0, "u0"), (d, "d"), (out, "out")]:
        if t is not None:
            _, h2, w2, ld2 = _img(t, n)
            if (h2, w2, ld2) != (h, w, ld) or t.dtype != torch.float32:
                raise ValueError(f"{n} must match f in shape, pitch and dtype")
    lib = load()
    if workspace is None:
        workspace = _workspace(lib.wmc_denoise_l1_workspace_size(h, w, ld), f.device)
    _check(lib.wmc_denoise_l1(p, u0.data_ptr() if u0 is not None else None, out.data_ptr(),
                              d.data_ptr() if d is not None else None, h, w, ld, float(lam), float(step),
                              float(alpha), int(iters), BOUNDARY[boundary], workspace.data_ptr(),
                              workspace.numel(), _stream(f.device)), "wmc_denoise_l1")
    return out


def _stack(t: torch.Tensor, name: str):
    """(ptr, n, h, w, ld) of an FP32 (n, h, w) CUDA tensor whose image i starts at i*h*ld."""
    if not t.is_cuda or t.dtype != torch.float32 or t.dim() != 3:
        raise ValueError(f"{name} must be a float32 CUDA tensor of shape (n, h, w)")
    n, h, w = t.shape
    ld = max(t.stride(1), w) if h > 1 else w
    if t.stride(2) != 1 or (h > 1 and t.stride(1) < w) or (n > 1 and t.stride(0) != h * ld):
        raise ValueError(f"{name}: rows must have unit stride and images a stride of h * ld")
    return t.data_ptr(), n, h, w, ld


def unrolled_workspace_size(n: int, h: int, w: int, K: int, ckpt_every: int, ld: int | None = None) -> int:
    return load().wmc_unrolled_workspace_size(n, h, w, w if ld is None else ld, K, ckpt_every)


def unrolled_forward(f: torch.Tensor, lam: torch.Tensor, step: float, K: int, ckpt_every: int = 7,
                     boundary: str = "replicate", out: torch.Tensor | None = None,
                     workspace: torch.Tensor | None = None):
    """U^K of K denoising steps of each image of the (n, h, w) stack f, lambda per image (a CUDA
    tensor of n floats).  Returns (U^K, workspace); the workspace holds the checkpoints that
    unrolled_backward needs."""
    pf, n, h, w, ld = _stack(f, "f")
    if lam.dtype != torch.float32 or lam.numel() != n or not lam.is_cuda or not lam.is_contiguous():
        raise ValueError("lam must be a contiguous float32 CUDA tensor with one value per image")
    lib = load()
    if out is None:
        out = torch.empty_strided(f.shape, f.stride(), dtype=f.dtype, device=f.device)
    po, n2, h2, w2, ld2 = _stack(out, "out")
    if (n2, h2, w2, ld2) != (n, h, w, ld):
        raise ValueError("out must match f in shape and pitch")
    if workspace is None:
        workspace = _workspace(lib.wmc_unrolled_workspace_size(n, h, w, ld, K, ckpt_every), f.device)
    _check(lib.wmc_unrolled_forward(pf, lam.data_ptr(), float(step), int(K), int(ckpt_every), n, h, w, ld,
                                    BOUNDARY[boundary], po, workspace.data_ptr(), workspace.numel(),
                                    _stream(f.device)), "wmc_unrolled_forward")
    return out, workspace


def unrolled_backward(f: torch.Tensor, lam: torch.Tensor, step: float, K: int, grad_u: torch.Tensor,
                      workspace: torch.Tensor, ckpt_every: int = 7, boundary: str = "replicate"):
    """(dL/df, dL/dlambda) from dL/dU^K, reading the checkpoints unrolled_forward left in
    `workspace` (selection held fixed)."""
    pf, n, h, w, ld = _stack(f, "f")
    grad_u = grad_u.contiguous() if f.is_contiguous() else grad_u
    pg, n2, h2, w2, ld2 = _stack(grad_u, "grad_u")
    if (n2, h2, w2, ld2) != (n, h, w, ld):
        raise ValueError("grad_u must match f in shape and pitch")
    grad_f = torch.empty_strided(f.shape, f.stride(), dtype=f.dtype, device=f.device)
    grad_lam = torch.empty(n, dtype=torch.float32, device=f.device)
    _check(load().wmc_unrolled_backward(pf, lam.data_ptr(), float(step), int(K), int(ckpt_every), n, h, w,
                                        ld, BOUNDARY[boundary], pg, grad_f.data_ptr(), grad_lam.data_ptr(),
                                        workspace.data_ptr(), workspace.numel(), _stream(f.device)),
           "wmc_unrolled_backward")
    return grad_f, grad_lam


def backward(f: torch.Tensor, lam: torch.Tensor, step: float, K: int, grad_u: torch.Tensor, ckpt_every: int = 7,
             boundary: str = "replicate", workspace: torch.Tensor | None = None):
    """(dL/df, dL/dlambda) of K unrolled denoising steps from dL/dU^K in one call (wmc_backward:
    the forward sweep that stores the checkpoints, then the reverse sweep)."""
    pf, n, h, w, ld = _stack(f, "f")
    if lam.dtype != torch.float32 or lam.numel() != n or not lam.is_cuda or not lam.is_contiguous():
        raise ValueError("lam must be a contiguous float32 CUDA tensor with one value per image")
    pg, n2, h2, w2, ld2 = _stack(grad_u, "grad_u")
    if (n2, h2, w2, ld2) != (n, h, w, ld):
        raise ValueError("grad_u must match f in shape and pitch")
    lib = load()
    if workspace is None:
        workspace = _workspace(lib.wmc_backward_workspace_size(n, h, w, ld, K, ckpt_every), f.device)
    grad_f = torch.empty_strided(f.shape, f.stride(), dtype=f.dtype, device=f.device)
    grad_lam = torch.empty(n, dtype=torch.float32, device=f.device)
    _check(lib.wmc_backward(pf, lam.data_ptr(), float(step), int(K), int(ckpt_every), n, h, w, ld,
                            BOUNDARY[boundary], pg, grad_f.data_ptr(), grad_lam.data_ptr(), workspace.data_ptr(),
                            workspace.numel(), _stream(f.device)), "wmc_backward")
    return grad_f, grad_lam


class UnrolledDenoise(torch.autograd.Function):
    """Autograd node of K unrolled denoising steps: apply(f, lam, step, K, ckpt_every, boundary).

    f: (n, h, w) float32 CUDA stack; lam: (n,) float32 CUDA tensor.  Gradients flow to f and lam;
    the backward recomputes the steps between checkpoints (every `ckpt_every` steps)."""

    @staticmethod
    def forward(ctx, f, lam, step, K, ckpt_every=7, boundary="replicate"):
        f = f.contiguous()
        lam = lam.contiguous()
        u, ws = unrolled_forward(f, lam, step, K, ckpt_every, boundary)
        ctx.save_for_backward(f, lam)
        ctx.ws, ctx.step, ctx.K, ctx.c, ctx.bnd = ws, step, K, ckpt_every, boundary
        return u

    @staticmethod
    def backward(ctx, grad_u):
        f, lam = ctx.saved_tensors
        gf, gl = unrolled_backward(f, lam, ctx.step, ctx.K, grad_u.contiguous(), ctx.ws, ctx.c, ctx.bnd)
        return gf, gl, None, None, None, None


# the same autograd node under the library's short name
WMCDenoise = UnrolledDenoise


def unrolled_denoise(f: torch.Tensor, lam: torch.Tensor, step: float, K: int, ckpt_every: int = 7,
                     boundary: str = "replicate") -> torch.Tensor:
    """Differentiable K-step denoising of an (n, h, w) stack (or one (h, w) image)."""
    squeeze = f.dim() == 2
    if squeeze:
        f = f.unsqueeze(0)
    lam = lam.reshape(-1)
    u = UnrolledDenoise.apply(f, lam, step, K, ckpt_every, boundary)
    return u[0] if squeeze else u


def energy_grad(u: torch.Tensor, boundary: str = "replicate", out: torch.Tensor | None = None) -> torch.Tensor:
    """d/dU sum_p |H^w(U)(p)| (selection held fixed, sign(0) = 0), FP32."""
    p, h, w, ld = _img(u, "u")
    if u.dtype != torch.float32:
        raise ValueError("energy_grad supports float32 only")
    if out is None:
        out = torch.empty_strided(u.shape, u.stride(), dtype=u.dtype, device=u.device)
    po, h2, w2, ld2 = _img(out, "out")
    if (h2, w2, ld2) != (h, w, ld):
        raise ValueError("out must match u in shape and pitch")
    _check(load().wmc_energy_grad(p, po, h, w, ld, BOUNDARY[boundary], _stream(u.device)),
           "wmc_energy_grad")
    return out


def shard_lpt(costs, world: int):
    """Partition images over `world` ranks by their costs (longest first, each to the least
    loaded rank; the library's wmc_shard_lpt).  Returns (owner per image, total cost per rank).
    Host only: no GPU is needed."""
    n = len(costs)
    c = (ctypes.c_int64 * max(n, 1))(*[int(x) for x in costs])
    owner = (ctypes.c_int32 * max(n, 1))()
    loads = (ctypes.c_int64 * max(int(world), 1))()
    _check(load().wmc_shard_lpt(ctypes.cast(c, _vp), n, int(world), ctypes.cast(owner, _vp),
                                ctypes.cast(loads, _vp)), "wmc_shard_lpt")
    return [int(owner[i]) for i in range(n)], [int(loads[r]) for r in range(int(world))]


def measure_fma_rate(device=None, iters: int = 4096, reps: int = 5) -> float:
    """FP32 FMA lane-operations per second of the current GPU (wmc_probe_fma; an FMA counts once),
    best of `reps` timed launches of 8 CTAs per SM."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    lib = load()
    blocks = 8 * torch.cuda.get_device_properties(dev).multi_processor_count
    threads = lib.wmc_probe_fma_threads()
    out = torch.empty(blocks * threads, dtype=torch.float32, device=dev)
    st = _stream(dev)
    _check(lib.wmc_probe_fma(out.data_ptr(), blocks, iters, st), "wmc_probe_fma")  # warm-up
    best = None
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        _check(lib.wmc_probe_fma(out.data_ptr(), blocks, iters, st), "wmc_probe_fma")
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    if not bool(torch.isfinite(out).all()):
        raise WMCError(4, "wmc_probe_fma", "non-finite probe output")
    return blocks * threads * iters * 16 / (best * 1e-3)


def psnr(sse: float, n: int, peak: float = 1.0) -> float:
    """PSNR in dB from a sum of squared errors over n pixels (FP64, host)."""
    import math
    if sse <= 0:
        return float("inf")
    return 10.0 * math.log10(peak * peak * n / sse)
