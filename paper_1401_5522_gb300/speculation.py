"""Decision predictor for speculative panel work (not part of the paper's method).

The factorization logs 16 features per step (see ``luqr_mlp_forward`` in the C header)
together with the criterion's decision.  A 16-64-64-1 MLP is trained on those pairs by
the library's own CUDA kernels (``luqr_mlp_grad`` + ``luqr_mlp_adam``); the trained
parameters are handed back to ``luqr_factor`` (``speculate="mlp"``), which uses the
network's prediction to factor a predicted-QR panel on a copy while the exact criterion
runs.  The criterion still decides every step, so decisions and results do not depend
on the predictor; only the time does.

Host-side logic here is bookkeeping: batching, feature standardisation (folded into the
first layer after training) and accuracy counting.
"""
from __future__ import annotations

import numpy as np

from . import luqr

F, H = luqr.MLP_FEATURES, 64


def init_params(seed=0):
    """He-initialised weights, zero biases, in the library's parameter layout."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((H, F)) * np.sqrt(2.0 / F)
    W2 = rng.standard_normal((H, H)) * np.sqrt(2.0 / H)
    W3 = rng.standard_normal(H) * np.sqrt(2.0 / H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), W3,
                           np.zeros(1)]).astype(np.float32)


def fold_standardisation(params, mu, sigma):
    """Parameters that take raw features: W1' = W1 / sigma, b1' = b1 - W1' mu."""
    p = np.array(params, dtype=np.float64)
    W1 = p[:H * F].reshape(H, F) / sigma[None, :]
    b1 = p[H * F:H * F + H] - W1 @ mu
    p[:H * F] = W1.ravel()
    p[H * F:H * F + H] = b1
    return p.astype(np.float32)


def collect(runs, device="cuda"):
    """Factor each run and return (features [S,16] float32, labels [S] float32, 1 = LU).

    runs: iterable of dicts with keys A (column-major float64 CUDA tensor), nb, and any
    keyword of luqr.factor (criterion, alpha, inject, precision, tree ...)."""
    feats, labels = [], []
    for r in runs:
        kw = dict(r)
        A = kw.pop("A")
        nb = kw.pop("nb")
        h = luqr.factor(A, nb, log_features=True, **kw)
        try:
            f, _ = h.features()
            dec, _ = h.decisions()
        finally:
            h.close()
        ok = dec != luqr.DEC_ABORTED
        feats.append(f[ok])
        labels.append((dec[ok] == luqr.DEC_LU).astype(np.float32))
    return np.concatenate(feats), np.concatenate(labels)


def train(X, y, epochs=300, batch=256, lr=3e-3, seed=0, device="cuda", log=None):
    """Train the MLP on (X, y) with the library's kernels; returns (params, losses).

    Features are standardised for training and the returned parameters take raw
    features (the standardisation is folded into the first layer)."""
    import torch
    X = np.asarray(X, dtype=np.float64)
    mu = X.mean(axis=0)
    sigma = X.std(axis=0)
    sigma[sigma < 1e-6] = 1.0
    Xs = ((X - mu) / sigma).astype(np.float32)
    Xd = torch.from_numpy(Xs).to(device)
    yd = torch.from_numpy(np.asarray(y, dtype=np.float32)).to(device)
    params = torch.from_numpy(init_params(seed)).to(device)
    grad = torch.zeros_like(params)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device=device)
    rng = np.random.default_rng(seed + 1)
    S = Xd.shape[0]
    losses = []
    t = 0
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(S)).to(device)
        Xp, yp = Xd[perm].contiguous(), yd[perm].contiguous()
        loss.zero_()
        nbatch = 0
        for s0 in range(0, S, batch):
            xb, yb = Xp[s0:s0 + batch], yp[s0:s0 + batch]
            grad.zero_()
            luqr.mlp_grad(params, xb, yb, grad, loss)
            t += 1
            luqr.mlp_adam(params, grad, m, v, t, lr=lr)
            nbatch += 1
        losses.append(float(loss.item()) / nbatch)
        if log and (ep % 50 == 0 or ep == epochs - 1):
            log(f"epoch {ep}: loss {losses[-1]:.4f}")
    raw = fold_standardisation(params.cpu().numpy(), mu, sigma)
    return torch.from_numpy(raw).to(device), losses


def predict(params, X, device="cuda"):
    """Predicted labels (1 = LU) of raw features X with the library's forward kernel."""
    import torch
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(device)
    return (luqr.mlp_forward(params, Xd).cpu().numpy() > 0).astype(np.float32)


def repeat_previous(labels_per_run):
    """Predictions of the repeat-the-previous-decision rule (LU at step 0)."""
    out = []
    for lab in labels_per_run:
        lab = np.asarray(lab, dtype=np.float32)
        out.append(np.concatenate([[1.0], lab[:-1]]) if len(lab) else lab)
    return out
