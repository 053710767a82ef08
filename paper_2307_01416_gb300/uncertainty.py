"""Statistical uncertainty of a Monte Carlo dose by the batch method.

The paper runs every plan to about 0.5 % statistical uncertainty (Sec. 2.D.3,
Sec. 3.C) without defining the estimate.  The reading used here: the
histories are split into B independent batches of equal size (independent
Philox seeds, the same histories per spot in each); the dose is the mean of
the batch doses and its standard error the batches' standard deviation over
sqrt(B); sigma_rel is the mean of SE / D over the voxels whose dose is at
least `level` x the maximum (0.5: the high-dose region), both taken inside a
mask (tissue: dose-to-medium in air-like voxels is not a clinical quantity).
The standard error of a Monte Carlo mean falls as 1 / sqrt(histories), so a
plan at sigma_rel with N histories per spot reaches `target` with
N (sigma_rel / target)^2.

Host-side statistics on dose arrays only: no transport arithmetic.
"""
from __future__ import annotations

import math
from typing import Optional, Tuple

import numpy as np


def batch_sigma_rel(batch_doses: np.ndarray, mask: Optional[np.ndarray] = None,
                    level: float = 0.5) -> Tuple[float, int]:
    """(sigma_rel, voxels it averages over) of the mean of B >= 2 batch doses.

    batch_doses: (B, nvox), each row an independent estimate of the same dose
    (equal histories per batch).  mask: (nvox,) bool, voxels that count."""
    d = np.asarray(batch_doses, dtype=np.float64)
    if d.ndim != 2 or d.shape[0] < 2:
        raise ValueError("need at least two batches, shaped (B, nvox)")
    b = d.shape[0]
    mean = d.mean(axis=0)
    se = d.std(axis=0, ddof=1) / math.sqrt(b)
    m = np.ones(mean.shape, dtype=bool) if mask is None else np.asarray(mask, dtype=bool).ravel()
    if not np.any(m & (mean > 0.0)):
        raise ValueError("no voxel with dose inside the mask")
    dmax = mean[m].max()
    sel = m & (mean >= level * dmax) & (mean > 0.0)
    return float(np.mean(se[sel] / mean[sel])), int(sel.sum())


def histories_for_target(n_hist: np.ndarray, sigma_rel: float, target: float) -> Tuple[np.ndarray, float]:
    """Histories per spot that bring a plan at sigma_rel (with n_hist per
    spot) to `target`: every spot scaled by (sigma_rel / target)^2, rounded
    up, at least 1.  Returns (new n_hist, scale factor)."""
    if not (sigma_rel > 0.0 and target > 0.0):
        raise ValueError("sigma_rel and target must be positive")
    f = (sigma_rel / target) ** 2
    n = np.maximum(np.ceil(np.asarray(n_hist, dtype=np.float64) * f), 1.0).astype(np.int64)
    return n, f


def split_histories(n_hist: np.ndarray, n_batches: int) -> np.ndarray:
    """Histories per spot of one of n_batches equal batches (rounded up;
    spots without histories keep none)."""
    n = np.asarray(n_hist, dtype=np.int64)
    return np.where(n > 0, (n + n_batches - 1) // n_batches, 0)
