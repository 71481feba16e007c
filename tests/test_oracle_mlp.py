"""The FP64 MLP reference: its analytic gradient against central finite differences."""
import numpy as np

from oracle import mlp_oracle as M


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = M.init_params(1)
    X = rng.standard_normal((20, M.F))
    y = (rng.random(20) < 0.4).astype(float)
    L, g = M.loss_and_grad(p, X, y)
    assert abs(L - M.loss(p, X, y)) < 1e-14
    idx = rng.choice(M.NPARAMS, size=60, replace=False)
    for i in idx:
        e = np.zeros(M.NPARAMS)
        e[i] = 1e-6
        fd = (M.loss(p + e, X, y) - M.loss(p - e, X, y)) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_parameter_count_and_layout():
    assert M.NPARAMS == 16 * 64 + 64 + 64 * 64 + 64 + 64 + 1
    p = np.arange(M.NPARAMS, dtype=float)
    q = M.unpack(p)
    assert q["W1"][0, 1] == 1 and q["b1"][0] == 1024 and q["b3"][0] == M.NPARAMS - 1
