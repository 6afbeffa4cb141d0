"""Reference ghost-rejection network -- TEST INFRASTRUCTURE.

A 12 -> 32 -> 32 -> 1 perceptron (ReLU, ReLU, sigmoid) scores track
candidates; it is trained on candidates labelled by generator truth.  The
paper has no learned component (its first stage cuts on a simplified fit,
Sec. "HLT1 details and results"); this network is the learned form that the
project adds on top, with the plain chi2 cut kept as the baseline.

This module holds the float64 reference of the training arithmetic (forward,
binary cross-entropy with logits, analytic backward) that the CUDA training
kernels are checked against, and the layout of the float32 model blob shared
with the C++ oracle (``vo_mlp_logit``) and the library:

    mean[12], inv_std[12], W1[32][12], b1[32], W2[32][32], b2[32], W3[32], b3
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 12
HIDDEN = 32
N_WEIGHTS = HIDDEN * N_FEATURES + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1  # 1505 trainable
N_FLOATS = 2 * N_FEATURES + N_WEIGHTS  # 1529


def unpack(blob: np.ndarray):
    """Split a model blob (or a weight vector of N_WEIGHTS) into its arrays (views)."""
    b = np.asarray(blob)
    off = 0
    out = {}
    if b.size == N_FLOATS:
        out["mean"] = b[0:N_FEATURES]
        out["inv_std"] = b[N_FEATURES:2 * N_FEATURES]
        off = 2 * N_FEATURES
    elif b.size != N_WEIGHTS:
        raise ValueError("blob size")
    for name, shape in (("W1", (HIDDEN, N_FEATURES)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
                        ("W3", (HIDDEN,)), ("b3", (1,))):
        n = int(np.prod(shape))
        out[name] = b[off:off + n].reshape(shape)
        off += n
    return out


def forward(w: np.ndarray, X: np.ndarray):
    """float64 forward of normalised inputs X [N, 12] with weights w [N_WEIGHTS].
    Returns (logits [N], cache)."""
    p = unpack(np.asarray(w, np.float64))
    X = np.asarray(X, np.float64)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["W3"] + p["b3"][0]
    return z, (X, a1, h1, a2, h2)


def loss(z: np.ndarray, y: np.ndarray) -> float:
    """Mean binary cross-entropy of sigmoid(z) against labels y in {0, 1} (stable form)."""
    z = np.asarray(z, np.float64)
    return float(np.mean(np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def backward(w: np.ndarray, X: np.ndarray, y: np.ndarray) -> tuple[float, np.ndarray]:
    """Loss and its gradient with respect to the N_WEIGHTS trainable values."""
    p = unpack(np.asarray(w, np.float64))
    z, (X, a1, h1, a2, h2) = forward(w, X)
    n = len(y)
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / n          # dL/dz
    gW3 = h2.T @ dz
    gb3 = np.array([dz.sum()])
    d2 = np.outer(dz, p["W3"]) * (a2 > 0)
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ p["W2"]) * (a1 > 0)
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])
    return loss(z, y), g


def pack(mean, inv_std, w) -> np.ndarray:
    return np.concatenate([np.asarray(mean, np.float32), np.asarray(inv_std, np.float32),
                           np.asarray(w, np.float32)]).astype(np.float32)
