"""Decision predictor on the GPU: the MLP kernels against the FP64 oracle, the logged
features against the oracle's factorization state, speculation leaving decisions and
results unchanged, and what the trained network gains over the plain method."""
import time

import numpy as np
import pytest
import torch

from oracle import luqr_oracle as O
from oracle import mlp_oracle as M
from paper_1401_5522_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1401_5522_gb300 import build
    build.build()


def L():
    from paper_1401_5522_gb300 import luqr
    return luqr


def dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def random_params(seed):
    rng = np.random.default_rng(seed)
    p = M.init_params(seed)
    p[1024:1088] = 0.1 * rng.standard_normal(64)      # nonzero biases exercise every term
    p[5184:5248] = 0.1 * rng.standard_normal(64)
    p[-1] = 0.05
    return p


@pytest.mark.parametrize("B", [1, 7, 256, 1000])
def test_forward_matches_oracle(B):
    rng = np.random.default_rng(B)
    p = random_params(1)
    X = rng.standard_normal((B, 16)) * 3.0
    z = L().mlp_forward(dev(p), dev(X)).cpu().numpy()
    ref = M.forward(p.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(z - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))


def test_forward_empty_batch():
    out = torch.empty(0, dtype=torch.float32, device="cuda")
    L().mlp_forward(dev(random_params(0)), torch.empty((0, 16), dtype=torch.float32, device="cuda"),
                    out)


@pytest.mark.parametrize("B", [1, 33, 777, 5000])
def test_gradient_matches_oracle(B):
    rng = np.random.default_rng(10 + B)
    p = random_params(2).astype(np.float32).astype(np.float64)
    X = (rng.standard_normal((B, 16)) * 2.0).astype(np.float32).astype(np.float64)
    y = (rng.random(B) < 0.5).astype(np.float64)
    grad = torch.zeros(M.NPARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    L().mlp_grad(dev(p), dev(X), dev(y), grad, loss)
    Lref, gref = M.loss_and_grad(p, X, y)
    g = grad.cpu().numpy()
    assert abs(loss.item() - Lref) <= 1e-5 * max(1.0, Lref)
    # FP32 accumulation over the batch: relative to the gradient's scale
    assert np.max(np.abs(g - gref)) <= 2e-5 * np.max(np.abs(gref)), np.max(np.abs(g - gref))


def test_adam_matches_oracle():
    rng = np.random.default_rng(5)
    p = rng.standard_normal(M.NPARAMS)
    m = np.zeros(M.NPARAMS)
    v = np.zeros(M.NPARAMS)
    dp, dm, dv = dev(p), dev(m), dev(v)
    for t in range(1, 6):
        g = rng.standard_normal(M.NPARAMS).astype(np.float32).astype(np.float64)
        p, m, v = M.adam_step(p, g, m, v, t, lr=1e-2)
        L().mlp_adam(dp, dev(g), dm, dv, t, lr=1e-2)
    assert np.max(np.abs(dp.cpu().numpy() - p)) <= 1e-5
    assert np.max(np.abs(dm.cpu().numpy() - m)) <= 1e-5
    assert np.max(np.abs(dv.cpu().numpy() - v)) <= 1e-5


def test_training_fits_a_separable_rule():
    from paper_1401_5522_gb300 import speculation as S
    rng = np.random.default_rng(7)
    X = rng.standard_normal((2000, 16)) * 4.0 + 3.0
    y = (X[:, 0] - 0.5 * X[:, 3] + 0.25 * X[:, 9] > 3.0).astype(np.float32)
    params, losses = S.train(X, y, epochs=60, batch=200, lr=3e-3)
    assert losses[-1] < 0.25 * losses[0]
    acc = np.mean(S.predict(params, X) == y)
    assert acc > 0.97, acc
    # the folded raw-feature network equals the oracle's forward on the same parameters
    z = L().mlp_forward(params, dev(X)).cpu().numpy()
    ref = M.forward(params.cpu().numpy().astype(np.float64), X.astype(np.float32))
    assert np.max(np.abs(z - ref)) <= 1e-3 * max(1.0, np.max(np.abs(ref)))


# ---------------------------------------------------------------- logged features

def test_features_match_oracle_state():
    # one injected panel keeps the trailing tiles well above rounding level (a second
    # 2^-27 scaling of the same rows would leave diagonal tiles of pure rounding noise)
    N, nb, alpha = 1024, 128, 4000.0
    A = inputs.gaussian(N, 11).numpy()
    inject = (3,)
    feats = []

    def hook(k, aug, fact):
        r0, r1 = k * nb, (k + 1) * nb
        norms = [O.norm1(aug[i * nb:(i + 1) * nb, r0:r1]) for i in range(k, fact.n)]
        away = (np.max(np.abs(aug[r1:N, r0:r1]), axis=0) if r1 < N else np.zeros(nb))
        feats.append(M.step_features(k, fact.n, alpha, O.CRIT_MAX, norms, aug[r0:r1, r0:r1], away,
                                     fact.dec[:k], fact.margin[:k]))

    f = O.factor(A, A @ np.ones(N), nb, O.CRIT_MAX, alpha, inject=inject, on_step=hook)
    h = L().factor(torch.from_numpy(np.asfortranarray(A)).cuda(), nb, "max", alpha, inject=inject,
                   log_features=True)
    dec, _ = h.decisions()
    fg, pred = h.features()
    h.close()
    assert np.array_equal(dec, f.dec)
    assert set(dec.tolist()) == {0, 1}
    ref = np.array(feats, dtype=np.float64)
    assert np.all(pred == L().DEC_ABORTED)
    err = np.abs(fg - ref) / np.maximum(1.0, np.abs(ref))
    assert np.max(err) <= 1e-5, err.max(axis=0)


# ---------------------------------------------------------------- speculation

def run(A, nb, criterion, alpha, **kw):
    luqr = L()
    b = inputs.ones_rhs(A)
    h = luqr.factor(A, nb, criterion, alpha, b=b, **kw)
    dec, mg = h.decisions()
    st = h.sync()
    W = h.factor_data()
    x = b.cpu().numpy()
    pred = h.features()[1] if kw.get("speculate", "off") != "off" else None
    h.close()
    return st, dec, mg, W, x, pred


@pytest.mark.parametrize("precision,tree", [("fp64", "flat_ts"), ("fp64", "binary_tt"),
                                            ("fp32", "binary_tt"), ("fp32", "grouped"),
                                            ("fp32", "flat_ts")])
def test_speculation_leaves_results_unchanged(precision, tree):
    N, nb = 2048 + 96, 128
    A = inputs.gaussian(N, 21, device="cuda")
    # one injected panel (more would push later diagonal tiles down to rounding level)
    inject = (3,)
    base = run(A, nb, "max", 4000.0, precision=precision, tree=tree, inject=inject)
    assert base[0] == 0 and set(base[1].tolist()) == {0, 1}
    params = dev(random_params(3))
    for mode, extra in (("repeat", {}), ("mlp", {"mlp_params": params})):
        got = run(A, nb, "max", 4000.0, precision=precision, tree=tree, inject=inject,
                  speculate=mode, **extra)
        assert got[0] == 0
        assert np.array_equal(got[1], base[1])
        assert np.array_equal(got[2], base[2])
        assert np.array_equal(got[3], base[3]), mode       # bit-identical factors
        assert np.array_equal(got[4], base[4]), mode       # and solution
        assert set(got[5].tolist()) <= {0, 1}
        if mode == "repeat":
            assert got[5][0] == 1 and np.array_equal(got[5][1:], base[1][:-1])


def test_speculation_all_qr_and_all_lu():
    N, nb = 1536, 128
    A = inputs.gaussian(N, 22, device="cuda")
    for crit, alpha in (("max", 0.0), ("force_lu", np.inf)):
        base = run(A, nb, crit, alpha, precision="fp64")
        got = run(A, nb, crit, alpha, precision="fp64", speculate="repeat")
        assert np.array_equal(got[1], base[1]) and np.array_equal(got[3], base[3])
        assert np.array_equal(got[4], base[4])


def test_speculation_rejects_missing_parameters():
    luqr = L()
    A = inputs.gaussian(256, 1, device="cuda")
    with pytest.raises(luqr.LuqrError):
        luqr.factor(A, 64, "max", 10.0, speculate="mlp")


def _time_factor(A, nb, reps=3, **kw):
    luqr = L()
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = luqr.factor(A, nb, **kw)
        h.sync()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
        h.close()
    return float(np.median(ts))


def test_trained_predictor_gain():
    """Train on 768 logged (features, decision) pairs from 48 small runs, then on held-out
    N = 16384 matrices whose decision sequences mix LU and QR irregularly: the MLP predicts
    the decisions better than the repeat-previous rule, and the factorization with MLP
    speculation (both predicted branches speculated) is faster than both the plain method
    and repeat-previous speculation, with the same decisions and bit-identical results."""
    from paper_1401_5522_gb300 import speculation as S
    nb = 256
    alphas = (1e4, 3e4, 1e5)

    def matrix(N, seed, frac):
        # iid N(0,1) with the diagonal tile of a fraction of the panels scaled by 1e-8
        A = inputs.gaussian(N, seed, device="cuda")
        return inputs.scale_diag_tiles(A, nb, inputs.choose_panels(N // nb, frac, seed), 1e-8)

    runs = [dict(A=matrix(4096, 100 + seed, 0.2), nb=nb, criterion="max", alpha=alphas[seed % 3],
                 precision="fp32", tree="binary_tt") for seed in range(48)]
    X, y = S.collect(runs)
    del runs
    assert len(y) == 768
    params, losses = S.train(X, y, epochs=200, batch=128, lr=3e-3)
    assert losses[-1] < losses[0]
    hits_mlp = hits_rep = total = 0
    t = {"off": 0.0, "repeat": 0.0, "mlp": 0.0}
    for seed, (frac, alpha) in enumerate(((0.2, 3e4), (0.4, 1e5))):
        A = matrix(16384, 900 + seed, frac)
        kw = dict(criterion="max", alpha=alpha, precision="fp32", tree="binary_tt")
        st, dec, mg, W0, x0, _ = run(A, nb, **kw)
        assert 0.2 < float(np.mean(dec)) < 0.8
        st1, dec1, mg1, W1, x1, pred = run(A, nb, speculate="mlp", mlp_params=params, **kw)
        assert np.array_equal(dec1, dec) and np.array_equal(W1, W0) and np.array_equal(x1, x0)
        hits_mlp += int(np.sum(pred == dec))
        hits_rep += int(np.sum(S.repeat_previous([dec])[0] == dec))
        total += len(dec)
        t["off"] += _time_factor(A, nb, **kw)
        t["repeat"] += _time_factor(A, nb, speculate="repeat", **kw)
        t["mlp"] += _time_factor(A, nb, speculate="mlp", mlp_params=params, **kw)
        del A, W0, W1
        torch.cuda.empty_cache()
    acc_mlp, acc_rep = hits_mlp / total, hits_rep / total
    print(f"\npredictor accuracy: mlp {acc_mlp:.3f}, repeat-previous {acc_rep:.3f}; factor time "
          f"off {t['off'] * 1e3:.1f} ms, repeat {t['repeat'] * 1e3:.1f} ms, "
          f"mlp {t['mlp'] * 1e3:.1f} ms")
    assert acc_mlp > acc_rep
    assert t["mlp"] < t["off"] and t["mlp"] < t["repeat"]
