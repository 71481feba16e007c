"""GPU (C interface) versus the CPU oracle, element by element on the same seeded inputs.

Bars (derivation in the design notes):
* decisions: identical sequences;
* normwise backward error of the GPU solution <= 1e-13 (FP64 runs);
* final triangle: max |U_gpu - U_oracle| <= TOL_U * max(1, rho) * max |U_oracle|, with
  rho = max |U_oracle| / max |A| the growth of the run (LU steps amplify rounding-order
  differences through their multipliers; QR steps do not);
* solution: max |x_gpu - x_oracle| <= TOL_X * max |x_oracle|;
* finite margins agree to 1e-9 (log2 units).
"""
import numpy as np
import pytest
import torch

from oracle import luqr_oracle as O
from paper_1401_5522_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_U = 1e-10
TOL_X = 1e-9
TOL_MARGIN = 1e-9


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1401_5522_gb300 import build
    build.build()


def L():
    from paper_1401_5522_gb300 import luqr
    return luqr


def cuda_colmajor(M):
    return torch.from_numpy(np.asfortranarray(M)).cuda()


def gpu_solve(A, b, nb, crit, alpha, **kw):
    luqr = L()
    dA = cuda_colmajor(A)
    db = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    h = luqr.factor(dA, nb, crit, alpha, b=db, **kw)
    dec, mg = h.decisions()
    st, step, row = h.info()
    x = db.cpu().numpy()
    return h, dec, mg, x, st


ORACLE_CRIT = {"max": O.CRIT_MAX, "sum": O.CRIT_SUM, "mumps": O.CRIT_MUMPS,
               "force_lu": O.CRIT_FORCE_LU, "force_qr": O.CRIT_FORCE_QR}
ORACLE_TREE = {"flat_ts": O.TREE_FLAT_TS, "binary_tt": O.TREE_BINARY_TT, "grouped": O.TREE_GROUPED}


def compare(A, nb, crit, alpha, tree="flat_ts", group=4, eta_bar=1e-13, **kw):
    N = A.shape[0]
    b = A @ np.ones(N)
    x_o, f = O.solve(A, b, nb, ORACLE_CRIT[crit], alpha, tree=ORACLE_TREE[tree], group=group, **kw)
    h, dec, mg, x_g, st = gpu_solve(A, b, nb, crit, alpha, tree=tree, group=group, **kw)
    assert st == 0, st
    assert np.array_equal(dec, f.dec), (dec, f.dec)
    fin = np.isfinite(f.margin)
    assert np.array_equal(np.isfinite(mg), fin)
    assert np.all(np.abs(mg[fin] - f.margin[fin]) <= TOL_MARGIN)
    eta = O.backward_error(A, x_g, b)
    assert eta <= eta_bar, eta
    assert np.max(np.abs(x_g - x_o.ravel())) <= TOL_X * np.max(np.abs(x_o))
    W = h.factor_data()
    Ug = np.triu(W[:N, :N])
    dU = np.max(np.abs(Ug - f.U))
    rho = np.max(np.abs(f.U)) / np.max(np.abs(A))
    assert dU <= TOL_U * max(1.0, rho) * np.max(np.abs(f.U)), (dU, rho)
    h.close()
    return f, dec, eta


def gauss(N, seed):
    return inputs.gaussian(N, seed).numpy()


# --------------------------------------------------- config 1: N=1024, nb=128, Max alpha=100
@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("crit,alpha", [("max", 100.0), ("force_lu", 0.0), ("force_qr", 0.0)])
def test_config1_parity(seed, crit, alpha):
    A = gauss(1024, seed)
    f, dec, eta = compare(A, 128, crit, alpha,
                          eta_bar=1e-13 if crit != "force_lu" else 1e-12)
    if crit == "max":
        assert list(dec) == [0] * 7 + [1]        # alpha = 100 is below every panel's need


@pytest.mark.parametrize("tree", ["flat_ts", "binary_tt", "grouped"])
@pytest.mark.parametrize("crit,alpha", [("max", 2000.0), ("sum", 6000.0), ("mumps", 2.1)])
def test_mixed_decisions_all_trees(tree, crit, alpha):
    A = gauss(512, 3)
    f, dec, _ = compare(A, 32, crit, alpha, tree=tree, group=3)


def test_mixed_sequence_really_mixes():
    A = gauss(512, 3)
    f, dec, _ = compare(A, 32, "max", 2000.0, tree="binary_tt")
    assert 0 < int(dec.sum()) < len(dec)


@pytest.mark.parametrize("N,nb", [(1000, 128), (333, 64), (65, 32)])
def test_ragged_sizes(N, nb):
    A = gauss(N, 4)
    compare(A, nb, "max", 3000.0, tree="binary_tt")
    compare(A, nb, "force_qr", 0.0, tree="flat_ts")


@pytest.mark.parametrize("nb", [32, 64, 256, 512])
def test_tile_sizes(nb):
    A = gauss(2 * nb + 17, 5)
    compare(A, nb, "max", 1e4, tree="binary_tt")


def test_worst_case_matrix_equality_on_gpu():
    n, nb, alpha = 6, 32, 2.0
    A = inputs.worst_case_max(n, nb, alpha).numpy()
    h, dec, mg, x, st = gpu_solve(A, A @ np.ones(n * nb), nb, "max", alpha)
    assert st == 0
    assert np.all(dec == 1)
    assert np.all(mg[:-1] == 0.0)             # Eq. 2 with equality, exact arithmetic
    lhs, rhs = h.step_stats()
    assert np.array_equal(lhs[:-1], rhs[:-1])
    W = h.factor_data()
    growth = np.max(np.abs(W)) / 1.0
    assert growth == (1.0 + alpha) ** (n - 1)


def test_block_diag_dominant_all_lu_on_gpu():
    A = inputs.block_diag_dominant(6, 32, seed=2).numpy()
    for crit in ("max", "sum"):
        h, dec, mg, x, st = gpu_solve(A, A @ np.ones(A.shape[0]), 32, crit, 1.0)
        assert np.all(dec == 1)


def test_forced_and_injected_steps():
    A = gauss(384, 6)
    forced = np.array([1, 0, 1, 1, 0, 1, 0, 1, 1, 0, 1, 1], dtype=np.uint8)
    compare(A + 30 * np.eye(384), 32, "max", 1.0, forced=forced, tree="binary_tt")
    N, nb = 256, 32
    A2 = gauss(N, 7) + 20 * np.eye(N)
    b = A2 @ np.ones(N)
    x_o, f = O.solve(A2, b, nb, O.CRIT_MAX, 1e6, inject=[2])
    h, dec, mg, x_g, st = gpu_solve(A2, b, nb, "max", 1e6, inject=[2])
    assert np.array_equal(dec, f.dec) and dec[2] == 0


def test_second_pass_solve_many_rhs():
    luqr = L()
    N, nb = 700, 64
    A = gauss(N, 8)
    B = np.random.default_rng(0).standard_normal((N, 3))
    for tree in ("flat_ts", "binary_tt", "grouped"):
        _, f = O.solve(A, None, nb, O.CRIT_MAX, 4000.0, tree=ORACLE_TREE[tree])
        X_o = O.replay_solve(f, B)
        h = luqr.factor(cuda_colmajor(A), nb, "max", 4000.0, tree=tree)
        dB = cuda_colmajor(B)
        h.solve(dB)
        X_g = dB.cpu().numpy()
        assert np.max(np.abs(X_g - X_o)) <= TOL_X * np.max(np.abs(X_o))
        for j in range(3):
            assert O.backward_error(A, X_g[:, j], B[:, j]) <= 1e-13


def test_nonfinite_and_singular_reported():
    luqr = L()
    A = gauss(128, 9)
    A[70, 3] = np.nan
    h = luqr.factor(cuda_colmajor(A), 32, "max", 10.0)
    st, step, row = h.info()
    assert st == luqr.ERR_NONFINITE and step == 0
    B = gauss(128, 9)
    B[32:64, 32:64] = 0.0
    B[32:64, :32] = 0.0
    h = luqr.factor(cuda_colmajor(B), 32, "force_lu", 0.0)
    st, step, row = h.info()
    assert st == luqr.ERR_SINGULAR and step == 1


# --------------------------------------------------- Hager-Higham estimate (norm_mode = 1)
@pytest.mark.parametrize("precision,crit,alpha", [("fp64", "max", 3000.0), ("fp64", "sum", 20000.0),
                                                  ("fp32", "max", 3000.0)])
def test_norm_estimate_matches_oracle(precision, crit, alpha):
    """The GPU estimator (FP64 arithmetic on the stored factors, blocked solves) against the
    oracle's: identical decisions, margins to 1e-9 (rounding order of the solves), and
    never a smaller margin than the exact norm at step 0 (same tile, lower-bound norm)."""
    N, nb = 1024, 64
    A = gauss(N, 31)
    b = A @ np.ones(N)
    dt = np.float32 if precision == "fp32" else np.float64
    _, f = O.solve(A, b, nb, ORACLE_CRIT[crit], alpha, dtype=dt, norm_mode=1)
    luqr = L()
    h = luqr.factor(cuda_colmajor(A), nb, crit, alpha, precision=precision, norm_mode="estimate")
    dec, mg = h.decisions()
    h.close()
    assert np.array_equal(dec, f.dec)
    assert set(dec.tolist()) == {0, 1}
    fin = np.isfinite(f.margin)
    tol = 1e-9 if precision == "fp64" else 1e-2
    assert np.all(np.abs(mg[fin] - f.margin[fin]) <= tol)
    h0 = luqr.factor(cuda_colmajor(A), nb, crit, alpha, precision=precision)
    _, mg0 = h0.decisions()
    h0.close()
    assert mg[0] >= mg0[0] - 1e-9


@pytest.mark.parametrize("seed", [0, 17])
def test_random_criterion_matches_oracle(seed):
    """Random choice (Sec. V-B): LU with probability alpha/100 per step from SplitMix64
    draws computed independently on both sides; identical decisions and margins, and a
    backward error within the LU-step bar."""
    N, nb = 1024, 64
    A = gauss(N, 40 + seed)
    b = A @ np.ones(N)
    _, f = O.solve(A, b, nb, O.CRIT_RANDOM, 50.0, seed=seed)
    h, dec, mg, x, st = gpu_solve(A, b, nb, "random", 50.0, seed=seed)
    h.close()
    assert st == 0
    assert np.array_equal(dec, f.dec)
    assert set(dec.tolist()) == {0, 1}
    assert np.all(np.abs(mg - f.margin) <= 1e-9)
    assert O.backward_error(A, x, b) <= 1e-12


def test_norm_mode_out_of_range_rejected():
    luqr = L()
    A = cuda_colmajor(gauss(128, 1))
    with pytest.raises(luqr.LuqrError):
        luqr.factor(A, 32, "max", 10.0, norm_mode=2)


# --------------------------------------------------- FP32 factorization + FP64 refinement
def test_fp32_decisions_match_float32_oracle():
    A = gauss(512, 10)
    b = A @ np.ones(512)
    _, f = O.solve(A, b, 64, O.CRIT_MAX, 3000.0, dtype=np.float32)
    luqr = L()
    h = luqr.factor(cuda_colmajor(A), 64, "max", 3000.0, precision="fp32")
    dec, mg = h.decisions()
    assert np.array_equal(dec, f.dec)
    fin = np.isfinite(f.margin)
    # FP32 rounding-order differences (~6e-8 relative) reach the margin through
    # ||A_kk^-1||_1, i.e. amplified by kappa(A_kk) ~ 1e3..1e4 on random tiles
    assert np.all(np.abs(mg[fin] - f.margin[fin]) <= 1e-2)


@pytest.mark.parametrize("tree,nb,kernels", [("binary_tt", 64, "tensor"), ("flat_ts", 64, "cuda"),
                                             ("grouped", 128, "tensor"), ("binary_tt", 256, "cuda"),
                                             ("flat_ts", 128, "tensor")])
def test_fp32_qr_factor_matches_float32_oracle(tree, nb, kernels):
    """All-QR FP32 runs (no pivot choice can flip, no growth) against the oracle's float32
    emulation, triangle element by element.  Rounding-order differences of FP32 sums (and
    the 3xTF32 operand split, ~2^-22 relative) stay within 2e-4 of max |U|."""
    N = 768 + 40
    A = gauss(N, 13)
    b = A @ np.ones(N)
    _, f = O.solve(A, b, nb, O.CRIT_FORCE_QR, 0.0, tree=ORACLE_TREE[tree], group=3,
                   dtype=np.float32)
    luqr = L()
    h = luqr.factor(cuda_colmajor(A), nb, "force_qr", 0.0, precision="fp32", tree=tree, group=3,
                    fp32_kernels=kernels)
    U = np.triu(h.factor_data()[:N, :N]).astype(np.float64)
    h.close()
    Uo = np.asarray(f.U, dtype=np.float64)
    assert np.max(np.abs(U - Uo)) <= 2e-4 * np.max(np.abs(Uo)), np.max(np.abs(U - Uo))


@pytest.mark.parametrize("tree,nb", [("flat_ts", 128), ("binary_tt", 128), ("binary_tt", 512),
                                     ("grouped", 256)])
def test_fp32_refinement_reaches_fp64_accuracy(tree, nb):
    luqr = L()
    N = 1024 if nb < 512 else 1536 + 40
    A = gauss(N, 11)
    dA = cuda_colmajor(A)
    b = torch.from_numpy(A @ np.ones(N)).cuda()
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    h = luqr.factor(dA, nb, "max", 100.0, precision="fp32", tree=tree)
    st, iters, eta = h.refine(dA, b, x, tol=1e-14, max_iter=20)
    assert st == 0, (st, iters, eta)
    assert eta <= 1e-14
    assert O.backward_error(A, x.cpu().numpy(), b.cpu().numpy()) <= 1e-13


@pytest.mark.parametrize("tree,crit,alpha,dd", [("binary_tt", "max", 100.0, False),
                                                ("grouped", "force_qr", 0.0, False),
                                                ("flat_ts", "force_lu", 0.0, True),
                                                ("flat_ts", "max", 3000.0, False),
                                                ("grouped", "sum", 8000.0, False)])
def test_fp32_tensor_core_updates_match_cuda_core_updates(tree, crit, alpha, dd):
    """The tcgen05 (3xTF32) trailing updates and the CUDA-core ones compute the same FP32
    factorization up to rounding: identical decisions and refinement to 1e-14 everywhere;
    U compared element-wise where no pivot choice can flip (QR-only runs, and all-LU on a
    diagonally dominant matrix).  In mixed runs a near-tie in a later GETRF's pivot search
    can pick the other row under a 1e-6 perturbation: a different, equally valid U."""
    luqr = L()
    N, nb = 768, 64
    A = gauss(N, 12) + (4.0 * np.sqrt(N) * np.eye(N) if dd else 0.0)
    dA = cuda_colmajor(A)
    h1 = luqr.factor(dA, nb, crit, alpha, precision="fp32", tree=tree, group=3,
                     fp32_kernels="tensor")
    h2 = luqr.factor(dA, nb, crit, alpha, precision="fp32", tree=tree, group=3,
                     fp32_kernels="cuda")
    d1, _ = h1.decisions()
    d2, _ = h2.decisions()
    assert np.array_equal(d1, d2)
    if crit in ("force_qr", "force_lu") or np.all(d1[:-1] == 0):
        U1 = np.triu(h1.factor_data()[:N, :N])
        U2 = np.triu(h2.factor_data()[:N, :N])
        rho = max(1.0, np.max(np.abs(U2)) / np.max(np.abs(A)))
        assert np.max(np.abs(U1 - U2)) <= 2e-4 * rho * np.max(np.abs(U2))
    b = torch.from_numpy(A @ np.ones(N)).cuda()
    for h in (h1, h2):
        x = torch.zeros(N, dtype=torch.float64, device="cuda")
        st, iters, eta = h.refine(dA, b, x, tol=1e-14, max_iter=20)
        assert st == 0 and eta <= 1e-14, (st, iters, eta)


@pytest.mark.parametrize("big,small,switch", [("binary_tt", "flat_ts", 6),
                                              ("grouped", "binary_tt", 4),
                                              ("flat_ts", "grouped", 10)])
@pytest.mark.parametrize("crit,alpha", [("max", 2000.0), ("force_qr", 0.0)])
def test_per_step_tree_policy_matches_oracle(big, small, switch, crit, alpha):
    """A tree that changes at a step (the small tree once fewer than `switch` sub-diagonal
    tiles remain) against the oracle with the same policy: decisions, margins, triangle,
    solution at the usual bars."""
    A = gauss(544, 5)
    N, nb = A.shape[0], 32
    b = A @ np.ones(N)
    x_o, f = O.solve(A, b, nb, ORACLE_CRIT[crit], alpha, tree=ORACLE_TREE[big], group=3,
                     tree_small=ORACLE_TREE[small], tree_switch=switch)
    h, dec, mg, x_g, st = gpu_solve(A, b, nb, crit, alpha, tree=big, group=3,
                                    tree_small=small, tree_switch=switch)
    assert st == 0, st
    assert np.array_equal(dec, f.dec), (dec, f.dec)
    fin = np.isfinite(f.margin)
    assert np.all(np.abs(mg[fin] - f.margin[fin]) <= TOL_MARGIN)
    assert O.backward_error(A, x_g, b) <= 1e-13
    assert np.max(np.abs(x_g - x_o.ravel())) <= TOL_X * np.max(np.abs(x_o))
    Ug = np.triu(h.factor_data()[:N, :N])
    rho = np.max(np.abs(f.U)) / np.max(np.abs(A))
    assert np.max(np.abs(Ug - f.U)) <= TOL_U * max(1.0, rho) * np.max(np.abs(f.U))
    b2 = gauss(N, 6)[:, 0].copy()
    y_o = O.replay_solve(f, b2).ravel()
    x2 = torch.from_numpy(b2.copy()).cuda()
    h.solve(x2)
    assert h.sync() == 0
    h.close()
    assert np.max(np.abs(x2.cpu().numpy() - y_o)) <= TOL_X * np.max(np.abs(y_o))


def test_tree_policy_rejects_bad_values():
    luqr = L()
    dA = cuda_colmajor(np.eye(64))
    for kw in (dict(tree_switch=-1), dict(tree_small=3, tree_switch=2)):
        with pytest.raises(luqr.LuqrError) as e:
            luqr.factor(dA, 32, "max", 100.0, **kw)
        assert e.value.status == luqr.ERR_INVALID


def test_tree_autotuner_picks_a_candidate_and_matches_the_oracle():
    from paper_1401_5522_gb300 import autotune
    luqr = L()
    A = gauss(1024, 8)
    dA = cuda_colmajor(A)
    pols = [("binary_tt", "flat_ts", 0, 4), ("binary_tt", "flat_ts", 8, 4),
            ("grouped", "binary_tt", 4, 3)]
    best, table = autotune.tune_tree(dA, 64, "max", 2000.0, policies=pols)
    assert best in pols and [p for p, _ in table] == pols
    assert all(ms > 0 for _, ms in table)
    for p in pols:   # each policy against the oracle run with the same policy
        h = luqr.factor(dA, 64, "max", 2000.0, tree=p[0], tree_small=p[1], tree_switch=p[2],
                        group=p[3])
        dec = h.decisions()[0]
        h.close()
        f = O.factor(A, None, 64, O.CRIT_MAX, 2000.0, tree=ORACLE_TREE[p[0]],
                     tree_small=ORACLE_TREE[p[1]], tree_switch=p[2], group=p[3])
        assert np.array_equal(dec, f.dec), (p, dec, f.dec)
