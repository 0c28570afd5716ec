"""Oracle: the 4D-TV regulariser (Sec. III-E) and its gradient, in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

R_4D-TV = lambda_s R_spatial(dsigma_i) + lambda_t R_temporal({dsigma_j}_{j<i}, dsigma_i),
added to the data term with weight lambda_TV (Eq. 13).  Readings:
* R_spatial = (1/V) sum over voxels of sqrt(d_p^2 + d_r^2 + d_c^2 + eps) with forward
  differences along the three axes; a difference that would leave the grid is 0.
* R_temporal = (1 / sum_j alpha_j) sum_j alpha_j sum over voxels sqrt((dsigma_i -
  dsigma_j)^2 + eps), alpha_j = exp(-(i - j)); 0 when there is no earlier frame.
* eps is not given by the paper; 1e-8 is used.
* lambda_TV = 0.002, lambda_s = 1, lambda_t = 0.1 (Sec. IV-D).
"""
from __future__ import annotations

import numpy as np

LAMBDA_TV = 0.002
LAMBDA_S = 1.0
LAMBDA_T = 0.1
TV_EPS = 1e-8


def _diffs(s):
    """Forward differences along (z, y, x) of a (Z, Y, X) volume, 0 at the far faces."""
    d = []
    for ax in range(3):
        a = np.zeros_like(s)
        sl_hi = [slice(None)] * 3
        sl_lo = [slice(None)] * 3
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(0, -1)
        a[tuple(sl_lo)] = s[tuple(sl_hi)] - s[tuple(sl_lo)]
        d.append(a)
    return d


def spatial(dsigma, dims, eps=TV_EPS):
    """(R_spatial, dR/d dsigma) for a length-V vector on a grid of (Z, Y, X) = dims."""
    s = np.asarray(dsigma, np.float64).reshape(dims)
    V = s.size
    d = _diffs(s)
    mag = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2 + eps)
    g = np.zeros_like(s)
    for ax in range(3):
        q = d[ax] / mag                  # d mag / d (its own difference)
        g -= q                           # difference = s[next] - s[self]
        sl_hi = [slice(None)] * 3
        sl_lo = [slice(None)] * 3
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(0, -1)
        g[tuple(sl_hi)] += q[tuple(sl_lo)]
    return float(mag.sum()) / V, g.reshape(-1) / V


def temporal(dsigma, previous, eps=TV_EPS):
    """(R_temporal, gradient) against the earlier outputs ``previous`` (oldest first)."""
    s = np.asarray(dsigma, np.float64)
    i = len(previous)
    if i == 0:
        return 0.0, np.zeros_like(s)
    alpha = np.exp(-(i - np.arange(i, dtype=np.float64)))
    val, g = 0.0, np.zeros_like(s)
    for a, p in zip(alpha, previous):
        diff = s - np.asarray(p, np.float64)
        mag = np.sqrt(diff * diff + eps)
        val += a * mag.sum()
        g += a * diff / mag
    return val / alpha.sum(), g / alpha.sum()


def regulariser(dims, previous, lam=LAMBDA_TV, lam_s=LAMBDA_S, lam_t=LAMBDA_T, eps=TV_EPS):
    """Callback ``reg(dsigma) -> (lam * R_4D-TV, gradient)`` for ``oracle.dip.dip_step``."""
    def reg(ds):
        vs, gs = spatial(ds, dims, eps)
        vt, gt = temporal(ds, previous, eps)
        return lam * (lam_s * vs + lam_t * vt), lam * (lam_s * gs + lam_t * gt)
    return reg
