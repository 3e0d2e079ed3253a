"""Tie-aware comparison of GPU results with the FP64 oracle.

H^w picks the candidate d_i of smallest magnitude (Eq. act).  When two candidates have
(nearly) equal magnitude, FP32 and FP64 may legitimately pick different ones -- and for an
opposite-sign pair the two values differ by 2|d|.  So the check is: for every pixel the GPU
value must lie within `tol` of SOME candidate whose magnitude is within `tau` of the
minimum.  Pixels where that set holds candidates of both signs are counted as ties.

Tolerances (written here, used by every parity test):
  TOL_REL = 1e-5  -- max abs error relative to the input range R = max(U) - min(U).  FP32
                     evaluation of the 9-tap sums carries a few ulp of 12*max|U| (about
                     1e-6 R); 1e-5 R leaves an order of magnitude of headroom.
  TAU_REL = 2^-18 -- candidates within 3.8e-6 R of the minimum magnitude count as tied:
                     several times the FP32 error of a candidate, so an FP32 argmin can only
                     differ from the FP64 one inside this band.
"""
import numpy as np

TOL_REL = 1e-5
TAU_REL = 2.0 ** -18


def tie_check(gpu, cand, R, tol_rel=TOL_REL, tau_rel=TAU_REL, transform=None, extra_tol=None):
    """gpu: (...,) values; cand: (..., 8) oracle candidates d_i.  `transform` maps candidate
    values to the compared quantity (e.g. one flow update); `extra_tol` adds a per-pixel
    allowance (storage rounding).  Returns (ok_mask, n_ties, max_err)."""
    gpu = np.asarray(gpu, dtype=np.float64)
    cand = np.asarray(cand, dtype=np.float64)
    mags = np.abs(cand)
    mn = mags.min(-1, keepdims=True)
    in_set = mags <= mn + tau_rel * R
    vals = transform(cand) if transform is not None else cand
    err = np.abs(vals - gpu[..., None])
    err = np.where(in_set, err, np.inf).min(-1)
    tol = tol_rel * R
    if extra_tol is not None:
        tol = tol + extra_tol
    ok = err <= tol
    pos = np.where(in_set, cand > 0, False).any(-1)
    neg = np.where(in_set, cand < 0, False).any(-1)
    ties = int((pos & neg).sum())
    return ok, ties, float(err.max()) if err.size else 0.0


def value_range(u):
    u = np.asarray(u, dtype=np.float64)
    r = float(u.max() - u.min()) if u.size else 0.0
    return r if r > 0 else 1.0
