"""FP64 CPU oracle for the Weighted Mean Curvature stencil and the flows built on it.

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline leg of the
benchmark use this package; the CUDA library never does, and this package never imports the
library.  The arithmetic lives in ``wmc_oracle.c`` (plain C, FP64, written from the paper's
definitions: the half-window kernels of Sec. IV-B, Eq. conv, Eq. act, the gradient flow of
Sec. V-B, Eq. MCF, the primal-dual update of Sec. V-C, the regulariser of Eq. wmcr, and the
conventional finite-difference discretisation of Eq. rhs that Sec. V-D compares against).  This
module only compiles it with gcc and marshals numpy arrays in and out.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wmc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

REPLICATE = 0
ZERO = 1
STORAGE = {"f64": 0, "bf16": 1, "f16": 2, "f32": 3}

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_i8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile wmc_oracle.c into _build/liboracle.so (gcc, -O2, OpenMP if available)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, i64, d = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_get_threads.restype = ctypes.c_int
            lib.oracle_kernel.argtypes = [ctypes.c_int, _dp]
            lib.oracle_canonical_order.argtypes = [_ip]
            lib.oracle_round_storage.argtypes = [d, ctypes.c_int]
            lib.oracle_round_storage.restype = d
            lib.oracle_wmc_eval.argtypes = [_dp, _dp, i32, i32, i64, i64, ctypes.c_int, _dp, _i8p]
            lib.oracle_wmc_flow.argtypes = [_dp, _dp, _dp, i32, i32, i64, d, d, i32, ctypes.c_int, d,
                                            ctypes.c_int]
            lib.oracle_energies.argtypes = [_dp, _dp, _dp, i32, i32, i64, ctypes.c_int, _dp]
            lib.oracle_wmc_l1_primal_dual.argtypes = [_dp, _dp, _dp, _dp, _dp, i32, i32, i64, d, d, d, i32,
                                                      ctypes.c_int]
            lib.oracle_energy_grad.argtypes = [_dp, i32, i32, ctypes.c_int, _dp]
            lib.oracle_fd_eval.argtypes = [_dp, _dp, i32, i32, i64, i64, ctypes.c_int]
            lib.oracle_fd_flow.argtypes = [_dp, _dp, _dp, i32, i32, i64, d, d, i32, ctypes.c_int, d]
            lib.oracle_unrolled_grad.argtypes = [_dp, _dp, i32, i32, d, d, i32, ctypes.c_int, _dp, _dp, _dp]
            lib.oracle_wmc_eval_points.argtypes = [_dp, i32, i32, i64, ctypes.c_int, _ip, _ip, i64, _dp,
                                                   _dp]
            lib.oracle_wmc_step_points.argtypes = [_dp, _dp, i32, i32, i64, d, d, d, ctypes.c_int, _ip,
                                                   _ip, i64, _dp, _dp]
            lib.oracle_count_ties.argtypes = [_dp, i32, i32, i64, ctypes.c_int, d, ctypes.POINTER(i64)]
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


def _bnd(boundary) -> int:
    if isinstance(boundary, str):
        return {"replicate": REPLICATE, "zero": ZERO}[boundary]
    return int(boundary)


def set_threads(n: int) -> None:
    """Split whole-image passes over n OpenMP threads (results do not depend on n)."""
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def kernel(i: int) -> np.ndarray:
    """h_{i+1} as the oracle stores it (3x3, FP64)."""
    out = np.zeros(9)
    _load().oracle_kernel(i, _ptr(out))
    return out.reshape(3, 3)


def canonical_order() -> list[int]:
    """0-based kernel indices in the order ties are resolved (first minimum wins)."""
    out = (ctypes.c_int32 * 8)()
    _load().oracle_canonical_order(out)
    return list(out)


def round_storage(x, storage: str) -> np.ndarray:
    """Round FP64 values to a storage format (bf16 / f16 / f32) and back, ties to even."""
    lib = _load()
    x = _f64(x)
    flat = x.ravel()
    out = np.fromiter((lib.oracle_round_storage(float(v), STORAGE[storage]) for v in flat),
                      dtype=np.float64, count=flat.size)
    return out.reshape(x.shape)


def wmc_eval(u, boundary="replicate", candidates: bool = False):
    """H^w of Eq. act for every pixel of a 2-D array.

    Returns hw, or (hw, cand, index) with cand[y, x, i] = d_{i+1} (Eq. conv) and index the
    selected kernel number 1..8.
    """
    u = _f64(u)
    h, w = u.shape
    hw = np.zeros((h, w))
    cand = np.zeros((h, w, 8)) if candidates else None
    index = np.zeros((h, w), dtype=np.uint8) if candidates else None
    rc = _load().oracle_wmc_eval(_ptr(u), _ptr(hw), h, w, w, w, _bnd(boundary), _ptr(cand),
                                 _ptr(index, _i8p))
    if rc:
        raise ValueError(f"oracle_wmc_eval failed ({rc})")
    return (hw, cand, index) if candidates else hw


def wmc_flow(f, lam: float, step: float, iters: int, boundary="replicate", mu: float = 1.0,
             u0=None, storage: str = "f64"):
    """`iters` Jacobi steps of U <- U + step*(lam*H^w(U) - mu*(U - f)) from U^0 = u0 (or f)."""
    ref = f if f is not None else u0
    ref = _f64(ref)
    h, w = ref.shape
    f_ = None if f is None else _f64(f)
    u0_ = None if u0 is None else _f64(u0)
    out = np.zeros((h, w))
    rc = _load().oracle_wmc_flow(_ptr(f_), _ptr(u0_), _ptr(out), h, w, w, float(lam), float(step),
                                 int(iters), _bnd(boundary), float(mu), STORAGE[storage])
    if rc:
        raise ValueError(f"oracle_wmc_flow failed ({rc})")
    return out


def denoise(f, lam: float, step: float, iters: int, boundary="replicate", u0=None,
            storage: str = "f64"):
    """L2 denoising gradient flow (Sec. V-B, A = I)."""
    return wmc_flow(f, lam, step, iters, boundary, 1.0, u0, storage)


def mcf(u0, step: float, iters: int, boundary="replicate"):
    """Mean-curvature flow U <- U + step*H^w(U) (Eq. MCF)."""
    return wmc_flow(None, 1.0, step, iters, boundary, 0.0, u0)


def energies(u, f=None, clean=None, boundary="replicate"):
    """(sum |H^w|, 1/2 sum (U-f)^2, sum (U-clean)^2) in FP64."""
    u = _f64(u)
    h, w = u.shape
    f_ = None if f is None else _f64(f)
    c_ = None if clean is None else _f64(clean)
    out = np.zeros(3)
    rc = _load().oracle_energies(_ptr(u), _ptr(f_), _ptr(c_), h, w, w, _bnd(boundary), _ptr(out))
    if rc:
        raise ValueError(f"oracle_energies failed ({rc})")
    return tuple(float(v) for v in out)


def l1_primal_dual(f, lam: float, step: float, alpha: float, iters: int, boundary="replicate",
                   u0=None, d0=None):
    """L1-fidelity primal-dual iteration of Sec. V-C from (U^0, d^0) = (u0 or f, d0 or 0);
    returns (U, d)."""
    f = _f64(f)
    h, w = f.shape
    u0_ = None if u0 is None else _f64(u0)
    d0_ = None if d0 is None else _f64(d0)
    out = np.zeros((h, w))
    d = np.zeros((h, w))
    rc = _load().oracle_wmc_l1_primal_dual(_ptr(f), _ptr(u0_), _ptr(d0_), _ptr(out), _ptr(d), h, w, w,
                                           float(lam), float(step), float(alpha), int(iters),
                                           _bnd(boundary))
    if rc:
        raise ValueError(f"oracle_wmc_l1_primal_dual failed ({rc})")
    return out, d


def eval_points(u, ys, xs, boundary="replicate", candidates: bool = False):
    """H^w at the listed pixels (any image size); optionally the eight d_i of each."""
    u = _f64(u)
    h, w = u.shape
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    n = ys.size
    out = np.zeros(n)
    cand = np.zeros((n, 8)) if candidates else None
    rc = _load().oracle_wmc_eval_points(_ptr(u), h, w, w, _bnd(boundary), _ptr(ys, _ip),
                                        _ptr(xs, _ip), n, _ptr(out), _ptr(cand))
    if rc:
        raise ValueError(f"oracle_wmc_eval_points failed ({rc})")
    return (out, cand) if candidates else out


def count_ties(u, tau: float, boundary="replicate") -> int:
    """Pixels whose candidates within `tau` of the smallest magnitude hold both signs (the
    opposite-sign near-ties of Eq. act)."""
    u = _f64(u)
    h, w = u.shape
    n = ctypes.c_int64(0)
    rc = _load().oracle_count_ties(_ptr(u), h, w, w, _bnd(boundary), float(tau), ctypes.byref(n))
    if rc:
        raise ValueError(f"oracle_count_ties failed ({rc})")
    return int(n.value)


def step_points(u, f, lam: float, step: float, ys, xs, boundary="replicate", mu: float = 1.0,
                candidates: bool = False):
    """One Jacobi update at the listed pixels, given U^t (and f when mu != 0)."""
    u = _f64(u)
    h, w = u.shape
    f_ = None if f is None else _f64(f)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    n = ys.size
    out = np.zeros(n)
    cand = np.zeros((n, 8)) if candidates else None
    rc = _load().oracle_wmc_step_points(_ptr(f_), _ptr(u), h, w, w, float(lam), float(step), float(mu),
                                        _bnd(boundary), _ptr(ys, _ip), _ptr(xs, _ip), n, _ptr(out),
                                        _ptr(cand))
    if rc:
        raise ValueError(f"oracle_wmc_step_points failed ({rc})")
    return (out, cand) if candidates else out


def unrolled_grad(f, clean, lam: float, step: float, K: int, boundary="replicate"):
    """Loss = mean((U^K - clean)^2) of K unrolled denoising steps from U^0 = f, and its gradient
    (dloss/dlambda, dloss/df) with each step's selection held fixed.  Returns (loss, dlam, df)."""
    f = _f64(f)
    clean = _f64(clean)
    h, w = f.shape
    loss = ctypes.c_double()
    dl = ctypes.c_double()
    df = np.zeros((h, w))
    rc = _load().oracle_unrolled_grad(_ptr(f), _ptr(clean), h, w, float(lam), float(step), int(K),
                                      _bnd(boundary), ctypes.byref(loss), ctypes.byref(dl), _ptr(df))
    if rc:
        raise ValueError(f"oracle_unrolled_grad failed ({rc})")
    return loss.value, dl.value, df


def unrolled_loss(f, clean, lam: float, step: float, K: int, boundary="replicate") -> float:
    """Forward only: mean((U^K - clean)^2)."""
    u = denoise(f, lam, step, K, boundary)
    return float(np.mean((u - _f64(clean)) ** 2))


def energy_grad(u, boundary="replicate"):
    """d(sum_p |H^w(U)(p)|)/dU with each pixel's selection held fixed (sign(0) = 0)."""
    u = _f64(u)
    h, w = u.shape
    g = np.zeros((h, w))
    rc = _load().oracle_energy_grad(_ptr(u), h, w, _bnd(boundary), _ptr(g))
    if rc:
        raise ValueError(f"oracle_energy_grad failed ({rc})")
    return g


def fd_eval(u, boundary="replicate"):
    """Finite-difference WMC of Eq. rhs (central differences; 0 where the gradient is zero)."""
    u = _f64(u)
    h, w = u.shape
    hw = np.zeros((h, w))
    rc = _load().oracle_fd_eval(_ptr(u), _ptr(hw), h, w, w, w, _bnd(boundary))
    if rc:
        raise ValueError(f"oracle_fd_eval failed ({rc})")
    return hw


def fd_flow(f, lam: float, step: float, iters: int, boundary="replicate", mu: float = 1.0, u0=None):
    """`iters` Jacobi steps of U <- U + step*(lam*H_fd(U) - mu*(U - f)) (f None: mean-curvature flow)."""
    ref = _f64(f if f is not None else u0)
    h, w = ref.shape
    f_ = None if f is None else _f64(f)
    u0_ = None if u0 is None else _f64(u0)
    out = np.zeros((h, w))
    rc = _load().oracle_fd_flow(_ptr(f_), _ptr(u0_), _ptr(out), h, w, w, float(lam), float(step), int(iters),
                                _bnd(boundary), float(mu))
    if rc:
        raise ValueError(f"oracle_fd_flow failed ({rc})")
    return out
