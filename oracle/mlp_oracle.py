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


def adam_step(p, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, Algorithm 1) at iteration t >= 1; returns (p, m, v)."""
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return np.asarray(p, dtype=np.float64) - lr * mhat / (np.sqrt(vhat) + eps), m, v


def _log2(v):
    return float(np.log2(max(float(v), 1e-300)))


def step_features(k, n, alpha, criterion, tile_norms, Akk, away_max, dec, margin):
    """The 16 predictor features of step k, from the state the criterion sees.

    tile_norms: ||A_ik||_1 for i = k..n-1 (Sec. III-D inputs); Akk: the diagonal tile;
    away_max[j]: max |A_ij| over the sub-diagonal tiles; dec, margin: the decisions and
    log2(lhs/rhs) margins of steps 0..k-1.  Definitions as in the C header.
    """
    Akk = np.abs(np.asarray(Akk, dtype=np.float64))
    local = Akk.max(axis=0)
    away = np.asarray(away_max, dtype=np.float64)
    diag = np.diag(Akk)
    lmax = local.max()
    ratio = np.where(local > 0, np.log2(np.maximum(away, 1e-300) / np.where(local > 0, local, 1.0)),
                     64.0)
    rest = np.asarray(tile_norms[1:], dtype=np.float64)

    def clamp(m):
        return 0.0 if np.isnan(m) else float(min(64.0, max(-64.0, m)))

    f = np.zeros(F)
    f[0] = _log2(tile_norms[0])
    f[1] = _log2(rest.max() if rest.size else 0.0)
    f[2] = _log2(rest.sum())
    f[3] = _log2(local.min())
    f[4] = _log2(diag.max() / max(lmax, 1e-300))
    f[5] = _log2(diag.min() / max(lmax, 1e-300))
    f[6] = clamp(ratio.max())
    f[7] = clamp(ratio.mean())
    f[8] = (1.0 if dec[k - 1] == 1 else 0.0) if k > 0 else 0.5
    f[9] = clamp(margin[k - 1]) if k > 0 else 0.0
    f[10] = clamp(margin[k - 2]) if k > 1 else 0.0
    f[11] = k / n
    f[12] = 64.0 if np.isinf(alpha) else _log2(alpha)
    f[13] = _log2(n - k)
    f[14] = criterion / 4.0
    f[15] = (np.sum(np.asarray(dec[:k]) == 0) / k) if k > 0 else 0.0
    return f
