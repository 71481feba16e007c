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


def test_zero_network_closed_forms():
    # all-zero parameters: every logit is 0, the loss is log 2 and only b3 and W3 see a
    # gradient through the (zero) hidden layers: d/db3 = mean(sigmoid(0) - y)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((7, M.F))
    y = np.array([1, 0, 1, 1, 0, 0, 1], dtype=float)
    L, g = M.loss_and_grad(np.zeros(M.NPARAMS), X, y)
    assert abs(L - np.log(2.0)) < 1e-15
    assert abs(g[-1] - np.mean(0.5 - y)) < 1e-15
    assert np.all(g[:-1] == 0.0)


def test_adam_first_step_is_signed_learning_rate():
    # at t = 1 the bias-corrected moments are g and g^2, so every parameter moves by
    # lr * g / (|g| + eps), i.e. lr * sign(g) for |g| >> eps (Kingma and Ba, Sec. 2)
    rng = np.random.default_rng(4)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    p1, m, v = M.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr=0.01)
    np.testing.assert_allclose(p - p1, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(p - p1, 0.01 * np.sign(g), rtol=1e-5)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-14)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-14)


def test_step_features_hand_computed():
    # identity diagonal tile, tile norms 1, 2, 4, sub-diagonal column maxima 2, two prior
    # steps (LU with margin 3, QR with margin -100), alpha 1024, MUMPS (id 2), k=2 of n=5
    f = M.step_features(2, 5, 1024.0, 2, [1.0, 2.0, 4.0], np.eye(4), [2.0] * 4,
                        np.array([1, 0], dtype=np.uint8), np.array([3.0, -100.0]))
    expect = [0.0, 2.0, np.log2(6.0), 0.0, 0.0, 0.0, 1.0, 1.0, 0.0, -64.0, 3.0, 0.4, 10.0,
              np.log2(3.0), 0.5, 0.5]
    np.testing.assert_allclose(f, expect, rtol=0, atol=1e-15)
    # a zero column in the diagonal tile: its away/local ratio saturates at 64
    A = np.eye(4)
    A[:, 1] = 0.0
    f0 = M.step_features(0, 3, np.inf, 0, [3.0, 1.0], A, [1.0] * 4, [], [])
    assert f0[6] == 64.0 and f0[8] == 0.5 and f0[12] == 64.0 and f0[15] == 0.0
    assert abs(f0[7] - 16.0) < 1e-15        # mean of 0, 64, 0, 0


def test_forward_of_a_hand_computed_sparse_network():
    """A network with a few non-zero weights, evaluated by hand.  Row = output unit in W1
    and W2, so a transposed W2 or a missing ReLU changes the logits below.
      x = (1, 0, 4, 0.5, 0...):  h1_0 = relu(2*1 - 0.5 + 0.5) = 2,  h1_1 = relu(4 - 3) = 1,
        h2_0 = relu(1.5*2 - 2*1 + 0.25) = 1.25,  h2_5 = relu(1*1) = 1,
        logit = 3*1.25 - 0.5*1 + 0.1 = 3.35
      x = (-1, 0, 1, 0, 0...):  h1_0 = relu(-2 + 0.5) = 0,  h1_1 = relu(1 - 3) = 0,
        h2_0 = relu(0.25) = 0.25,  h2_5 = 0,  logit = 3*0.25 + 0.1 = 0.85"""
    p = np.zeros(M.NPARAMS)
    q = M.unpack(np.arange(M.NPARAMS, dtype=float))          # offsets of every entry
    def at(name, *idx):
        return int(q[name][idx] if idx else q[name])
    p[at("W1", 0, 0)] = 2.0
    p[at("W1", 0, 3)] = -1.0
    p[at("b1", 0)] = 0.5
    p[at("W1", 1, 2)] = 1.0
    p[at("b1", 1)] = -3.0
    p[at("W2", 0, 0)] = 1.5
    p[at("W2", 0, 1)] = -2.0
    p[at("b2", 0)] = 0.25
    p[at("W2", 5, 1)] = 1.0
    p[at("W3", 0)] = 3.0
    p[at("W3", 5)] = -0.5
    p[at("b3", 0)] = 0.1
    X = np.zeros((2, M.F))
    X[0, [0, 2, 3]] = [1.0, 4.0, 0.5]
    X[1, [0, 2]] = [-1.0, 1.0]
    z = M.forward(p, X)
    assert abs(z[0] - 3.35) < 1e-14 and abs(z[1] - 0.85) < 1e-14, z
