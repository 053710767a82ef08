"""FP64 CPU oracle of the learned aperture surrogate's network.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): used by tests/ to check
the CUDA training and inference kernels.  It shares no code with the CUDA
path.

The surrogate is not in the paper.  It stands in for the in-brass stepping of
the aperture module (Sec. 2.B), which the paper reads from MCsquare-generated
distributions.  Here that role is taken by a small network.  Its definition
is stated once here, in plain numpy, in the order of its steps:

  input x (6 features of the proton at the block's entrance),
  h1 = relu(W1 x + b1)          W1: 128 x 6
  h2 = relu(W2 h1 + b2)         W2: 128 x 128
  z  = W3 h2 + b3               W3: 45 x 128
  z[0]            transmission logit
  z[1:5]          mixture logits alpha_c of 4 components
  z[5:25]         means mu_{c,j}      (component c = row of a 4 x 5 block)
  z[25:45]        log widths s_{c,j}  (sigma = exp(s)), diagonal Gaussians
                  over the 5 exit quantities y (energy loss, lateral offsets,
                  direction changes; see orc_surrogate_tracks).

Loss of one track with label t (1: it left through the exit plane) and
targets y:  softplus(z0) - t z0  +  t * ( -log sum_c pi_c N(y; mu_c, sigma_c^2) ),
pi = softmax(alpha); the batch loss is the mean.

BF16 emulation: the kernels hold x, W and h1, h2 in bfloat16 and sum in
FP32.  With bf16=True the forward rounds those operands to bfloat16
(round-to-nearest-even, from their FP32 value) and sums in FP64; the backward
rounds the GEMM operands dz, da2, da1 the same way.
"""
from __future__ import annotations

import math
from typing import Dict, Tuple

import numpy as np

D_IN, D_H, D_OUT = 6, 128, 45
N_COMP, D_Y = 4, 5
LOG_2PI = math.log(2.0 * math.pi)
S_MIN, S_MAX = -8.0, 4.0            # log-width clamp used when sampling


def bf16(x) -> np.ndarray:
    """Round to bfloat16, nearest-even, from the FP32 value; returned as FP64.
    bfloat16 keeps the top 16 bits of an IEEE binary32: adding 0x7FFF plus the
    lowest kept bit and truncating rounds half to even."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = a.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed: int = 0) -> Dict[str, np.ndarray]:
    """He-normal weights, zero biases (a CPU initialisation for tests)."""
    g = np.random.default_rng(seed)
    return {
        "W1": g.standard_normal((D_H, D_IN)) * math.sqrt(2.0 / D_IN), "b1": np.zeros(D_H),
        "W2": g.standard_normal((D_H, D_H)) * math.sqrt(2.0 / D_H), "b2": np.zeros(D_H),
        "W3": g.standard_normal((D_OUT, D_H)) * math.sqrt(1.0 / D_H) * 0.1, "b3": np.zeros(D_OUT),
    }


def _q(x, on: bool):
    return bf16(x) if on else np.asarray(x, dtype=np.float64)


def forward(P: Dict[str, np.ndarray], X: np.ndarray, bf16_ops: bool = True) -> Tuple[np.ndarray, dict]:
    """Network output z (B x 45) and the activations the backward needs."""
    x = _q(X, bf16_ops)
    W1, W2, W3 = (_q(P[k], bf16_ops) for k in ("W1", "W2", "W3"))
    a1 = x @ W1.T + P["b1"]
    h1 = _q(np.maximum(a1, 0.0), bf16_ops)
    a2 = h1 @ W2.T + P["b2"]
    h2 = _q(np.maximum(a2, 0.0), bf16_ops)
    z = h2 @ W3.T + P["b3"]
    return z, {"x": x, "a1": a1, "h1": h1, "a2": a2, "h2": h2, "W1": W1, "W2": W2, "W3": W3}


def split(z: np.ndarray):
    """(logit, alpha (B,4), mu (B,4,5), s (B,4,5)) views of z."""
    return z[:, 0], z[:, 1:5], z[:, 5:25].reshape(-1, N_COMP, D_Y), z[:, 25:45].reshape(-1, N_COMP, D_Y)


def _logsumexp(a: np.ndarray, axis: int) -> np.ndarray:
    m = np.max(a, axis=axis, keepdims=True)
    return (m + np.log(np.sum(np.exp(a - m), axis=axis, keepdims=True))).squeeze(axis)


def _softplus(v: np.ndarray) -> np.ndarray:
    return np.maximum(v, 0.0) + np.log1p(np.exp(-np.abs(v)))


def component_log_density(z: np.ndarray, y: np.ndarray) -> np.ndarray:
    """log pi_c + log N(y; mu_c, diag sigma_c^2) per track and component (B, 4)."""
    _, alpha, mu, s = split(z)
    logpi = alpha - _logsumexp(alpha, 1)[:, None]
    r = (y[:, None, :] - mu) * np.exp(-s)
    return logpi + np.sum(-0.5 * r * r - s - 0.5 * LOG_2PI, axis=2)


def loss_terms(z: np.ndarray, t: np.ndarray, y: np.ndarray):
    """Per-track (BCE, mixture NLL); the NLL is 0 where t = 0."""
    logit = z[:, 0]
    bce = _softplus(logit) - t * logit
    nll = np.where(t > 0, -_logsumexp(component_log_density(z, y), 1), 0.0)
    return bce, nll


def loss(z: np.ndarray, t: np.ndarray, y: np.ndarray) -> float:
    bce, nll = loss_terms(z, t, y)
    return float(np.mean(bce + t * nll))


def loss_grad(z: np.ndarray, t: np.ndarray, y: np.ndarray) -> np.ndarray:
    """d(mean loss)/dz, written out from the loss's definition:
    d/dz0 = sigmoid(z0) - t; with responsibilities r_c (posterior of c):
    d/dalpha_c = t (pi_c - r_c); d/dmu = -t r_c (y - mu) / sigma^2;
    d/ds = -t r_c ((y - mu)^2 / sigma^2 - 1)."""
    B = z.shape[0]
    logit, alpha, mu, s = split(z)
    g = np.zeros_like(z)
    g[:, 0] = 1.0 / (1.0 + np.exp(-logit)) - t
    lc = component_log_density(z, y)
    resp = np.exp(lc - _logsumexp(lc, 1)[:, None])
    pi = np.exp(alpha - _logsumexp(alpha, 1)[:, None])
    tt = t[:, None]
    g[:, 1:5] = tt * (pi - resp)
    inv2 = np.exp(-2.0 * s)
    diff = y[:, None, :] - mu
    g[:, 5:25] = (-tt[:, :, None] * resp[:, :, None] * diff * inv2).reshape(B, -1)
    g[:, 25:45] = (-tt[:, :, None] * resp[:, :, None] * (diff * diff * inv2 - 1.0)).reshape(B, -1)
    return g / B


def backward(cache: dict, dz: np.ndarray, bf16_ops: bool = True) -> Dict[str, np.ndarray]:
    """Parameter gradients from dz by the chain rule through the two ReLU
    layers; bias gradients are sums of the unrounded deltas."""
    dzq = _q(dz, bf16_ops)
    g = {"W3": dzq.T @ cache["h2"], "b3": dz.sum(0)}
    da2 = (dzq @ cache["W3"]) * (cache["a2"] > 0.0)
    da2q = _q(da2, bf16_ops)
    g["W2"] = da2q.T @ cache["h1"]
    g["b2"] = da2.sum(0)
    da1 = (da2q @ cache["W2"]) * (cache["a1"] > 0.0)
    da1q = _q(da1, bf16_ops)
    g["W1"] = da1q.T @ cache["x"]
    g["b1"] = da1.sum(0)
    return g


def adam_step(P: Dict[str, np.ndarray], G: Dict[str, np.ndarray], M: Dict[str, np.ndarray],
              V: Dict[str, np.ndarray], step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8) -> None:
    """One Adam update (Kingma & Ba 2015, Algorithm 1), in place; step >= 1."""
    for k in P:
        M[k] = beta1 * M[k] + (1.0 - beta1) * G[k]
        V[k] = beta2 * V[k] + (1.0 - beta2) * G[k] * G[k]
        mhat = M[k] / (1.0 - beta1 ** step)
        vhat = V[k] / (1.0 - beta2 ** step)
        P[k] = P[k] - lr * mhat / (np.sqrt(vhat) + eps)


def sample(z: np.ndarray, u: np.ndarray):
    """Draw from the network's output with given uniforms u (B x 8):
    transmitted = u0 < sigmoid(z0); component = first c with u1 < sum_{c'<=c} pi;
    normals from Box-Muller pairs (u2, u3), (u4, u5), (u6, u7) -> xi_0..xi_4;
    y_j = mu_cj + exp(clamp(s_cj, S_MIN, S_MAX)) xi_j.
    Returns (transmitted (B,), component (B,), y (B, 5))."""
    logit, alpha, mu, s = split(z)
    p = 1.0 / (1.0 + np.exp(-logit))
    trans = u[:, 0] < p
    pi = np.exp(alpha - _logsumexp(alpha, 1)[:, None])
    cum = np.cumsum(pi, axis=1)
    comp = np.minimum(np.sum(u[:, 1:2] >= cum, axis=1), N_COMP - 1)
    xi = np.empty((z.shape[0], 6))
    for k in range(3):
        r = np.sqrt(-2.0 * np.log(u[:, 2 + 2 * k]))
        xi[:, 2 * k] = r * np.cos(2.0 * math.pi * u[:, 3 + 2 * k])
        xi[:, 2 * k + 1] = r * np.sin(2.0 * math.pi * u[:, 3 + 2 * k])
    rows = np.arange(z.shape[0])
    y = mu[rows, comp] + np.exp(np.clip(s[rows, comp], S_MIN, S_MAX)) * xi[:, :5]
    return trans, comp, y
