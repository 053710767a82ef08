"""FP64 CPU oracle of the robust spot-weight optimisation over the scenarios'
influence matrices.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/).

The paper optimises robustly over 13 scenarios (Sec. 2.E: SPR x (1 +- 3 %),
isocentre shifts +-2 mm) against the target dose-volume constraints of its
Table 3 (V100 %, D_min, CI100 %, RHI100 %).  Its optimiser is an in-house
trial-and-error procedure whose objective is not given.  This oracle states
the reading used here, step by step:

  dose of scenario s:         d_s = A_s x            (A_s: voxels x spots, x >= 0)
  objective of a dose d:      f(d) = w_u/|T| sum_T max(0, D_p - d)^2
                                   + w_o/|T| sum_T max(0, d - o D_p)^2
                                   + w_r/|R| sum_R max(0, d - q D_p)^2
                              (T target voxels, R ring voxels around it)
  robust objective:           F(x) = max_s f(A_s x)          (worst case)
  one iteration:              s* = the first s with f_s = max; g = A_s*^T f'(d_s*);
                              Adam (beta 0.9 / 0.999, eps) on x; x <- max(x, 0)
  target indices of a dose:   V100 = fraction of T with d >= D_p; D_min = min_T d / D_p;
                              CI100 = |{d >= D_p}| / |T|; RHI100 = max_T d / D_p
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Sequence

import numpy as np


@dataclass
class OptParams:
    prescription: float             # D_p, dose units of A x
    w_under: float = 1.0
    w_over: float = 0.5
    w_ring: float = 0.2
    over_frac: float = 1.05         # o
    ring_frac: float = 0.6          # q
    lr: float = 0.05                # Adam step, in units of the initial mean weight
    eps: float = 1e-8


def objective(d: np.ndarray, cls: np.ndarray, p: OptParams):
    """(f, f'(d)) of one dose vector; cls 1 target, 2 ring, else ignored."""
    T, R = cls == 1, cls == 2
    nT, nR = max(int(T.sum()), 1), max(int(R.sum()), 1)
    u = np.where(T, np.maximum(0.0, p.prescription - d), 0.0)
    o = np.where(T, np.maximum(0.0, d - p.over_frac * p.prescription), 0.0)
    q = np.where(R, np.maximum(0.0, d - p.ring_frac * p.prescription), 0.0)
    f = p.w_under / nT * np.sum(u * u) + p.w_over / nT * np.sum(o * o) + p.w_ring / nR * np.sum(q * q)
    g = -2.0 * p.w_under / nT * u + 2.0 * p.w_over / nT * o + 2.0 * p.w_ring / nR * q
    return float(f), g


def robust_objective(mats: Sequence, x: np.ndarray, cls: np.ndarray, p: OptParams):
    """(F, per-scenario f, s*, the doses)."""
    doses = [np.asarray(A @ x, dtype=np.float64) for A in mats]
    fs = np.array([objective(d, cls, p)[0] for d in doses])
    s = int(np.argmax(fs))
    return float(fs[s]), fs, s, doses


def optimise(mats: Sequence, x0: np.ndarray, cls: np.ndarray, p: OptParams, iterations: int,
             trace: List | None = None):
    """Run the iterations; returns (x, worst-case objective before each step).
    trace, if given, receives every iteration's per-scenario objectives."""
    x = np.asarray(x0, dtype=np.float64).copy()
    m = np.zeros_like(x)
    v = np.zeros_like(x)
    scale = float(np.mean(x0)) if np.mean(x0) > 0 else 1.0
    hist = []
    for t in range(1, iterations + 1):
        F, fs, s, doses = robust_objective(mats, x, cls, p)
        hist.append(F)
        if trace is not None:
            trace.append(fs)
        _, r = objective(doses[s], cls, p)
        g = np.asarray(mats[s].T @ r, dtype=np.float64)
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        mhat = m / (1.0 - 0.9 ** t)
        vhat = v / (1.0 - 0.999 ** t)
        x = np.maximum(x - p.lr * scale * mhat / (np.sqrt(vhat) + p.eps), 0.0)
    return x, np.array(hist)


def target_indices(d: np.ndarray, cls: np.ndarray, prescription: float) -> Dict[str, float]:
    T = cls == 1
    dt = d[T]
    return {"V100": float(np.mean(dt >= prescription)), "Dmin": float(dt.min() / prescription),
            "CI100": float(np.sum(d >= prescription) / max(int(T.sum()), 1)),
            "RHI100": float(dt.max() / prescription)}
