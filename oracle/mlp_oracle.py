"""CPU FP64 reference of the decision-predicting MLP (16 -> 64 -> 64 -> 1, ReLU, logit).

TEST INFRASTRUCTURE ONLY (same rule as luqr_oracle): the GPU training kernels' forward
pass, loss and gradients are checked against these plain numpy formulas.  The network is
not part of the paper; it predicts the robustness test's outcome so that the predicted
branch's panel work can start early.

Parameter vector layout (float32 on the GPU, float64 here), length 5313:
  W1[64][16] (row-major), b1[64], W2[64][64], b2[64], W3[64], b3[1].
Loss: mean binary cross-entropy with logits, label 1 = LU step, 0 = QR step.
Parity status: pinned by finite differences of this same loss (test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np

F, H = 16, 64
SIZES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H,)), ("b3", (1,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    out, off = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[off:off + n], dtype=np.float64).reshape(shape)
        off += n
    return out


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in SIZES:
        if name.startswith("W"):
            fan_in = shape[-1] if len(shape) > 1 else H
            parts.append(rng.standard_normal(int(np.prod(shape))) * np.sqrt(2.0 / fan_in))
        else:
            parts.append(np.zeros(int(np.prod(shape))))
    return np.concatenate(parts)


def forward(p, X):
    """Logits for a batch X (B x 16)."""
    q = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ q["W1"].T + q["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ q["W2"].T + q["b2"]
    h2 = np.maximum(z2, 0.0)
    return h2 @ q["W3"] + q["b3"][0]


def loss(p, X, y):
    """Mean binary cross-entropy with logits."""
    z = forward(p, X)
    y = np.asarray(y, dtype=np.float64)
    return float(np.mean(np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def loss_and_grad(p, X, y):
    """(loss, gradient) by reverse-mode differentiation of the formulas above."""
    q = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    B = X.shape[0]
    z1 = X @ q["W1"].T + q["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ q["W2"].T + q["b2"]
    h2 = np.maximum(z2, 0.0)
    z = h2 @ q["W3"] + q["b3"][0]
    L = float(np.mean(np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))))
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / B
    gW3 = h2.T @ dz
    gb3 = np.array([dz.sum()])
    dz2 = np.outer(dz, q["W3"]) * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ q["W2"]) * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])
    return L, g
