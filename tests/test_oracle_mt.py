"""Pins of the threaded C++ oracle (oracle/luqr_oracle_mt.cpp), the one that runs the
benchmarked sizes.

It is checked against the pinned numpy oracle (same decisions, margins and transformed
matrix on mixed runs of every criterion and tree, ragged N, run-time injection, replayed
decisions, float32 storage), and directly against what the mathematics fixes: LAPACK
GEPP for one-tile FORCE_LU, numpy's Householder R for FORCE_QR on every tree, the
worst-case matrix of Sec. III-A (every step LU, margin exactly 0), block diagonal
dominance (Sec. III-B, all LU), x = 1 for b = A 1, and the independence of its results
from the thread count.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import luqr_oracle as O
from oracle import luqr_oracle_mt as M
from paper_1401_5522_gb300 import inputs


def gauss(N, seed):
    return np.random.default_rng(seed).standard_normal((N, N))


def check_same(fo, fm, tol_margin=1e-9, tol_aug=1e-10):
    assert np.array_equal(fo.dec, fm.dec), (fo.dec, fm.dec)
    fin = np.isfinite(fo.margin)
    assert np.array_equal(np.isfinite(fm.margin), fin)
    assert np.array_equal(np.sign(fo.margin[~fin]), np.sign(fm.margin[~fin]))
    if fin.any():
        assert np.max(np.abs(fo.margin[fin] - fm.margin[fin])) <= tol_margin
    rho = max(1.0, float(np.max(np.abs(fo.aug))))
    assert np.max(np.abs(fo.aug.astype(np.float64) - fm.aug.astype(np.float64))) <= tol_aug * rho


@pytest.mark.parametrize("tree", [O.TREE_FLAT_TS, O.TREE_BINARY_TT, O.TREE_GROUPED])
@pytest.mark.parametrize("crit,alpha,mode", [(O.CRIT_MAX, 2000.0, 0), (O.CRIT_SUM, 6000.0, 0),
                                             (O.CRIT_MUMPS, 2.1, 0), (O.CRIT_MUMPS, 3e5, 1),
                                             (O.CRIT_RANDOM, 50.0, 0)])
def test_same_run_as_numpy_oracle(tree, crit, alpha, mode):
    A = gauss(384, 3)
    b = A @ np.ones(384)
    kw = dict(tree=tree, group=3, mumps_mode=mode, seed=11)
    fo = O.factor(A, b, 32, crit, alpha, **kw)
    fm = M.factor(A, b, 32, crit, alpha, threads=3, **kw)
    check_same(fo, fm)
    assert 0 < int(fo.dec.sum()) < len(fo.dec)          # a mixed sequence
    fin = np.isfinite(fo.lhs)
    assert np.allclose(fm.lhs[fin], fo.lhs[fin], rtol=1e-9)
    assert np.allclose(fm.rhs[fin], fo.rhs[fin], rtol=1e-12)


@pytest.mark.parametrize("N,nb", [(333, 64), (65, 32), (100, 32)])
def test_ragged_injected_and_forced(N, nb):
    A = gauss(N, 4)
    b = A @ np.ones(N)
    n = (N + nb - 1) // nb
    fo = O.factor(A, b, nb, O.CRIT_MAX, 3000.0, tree=O.TREE_BINARY_TT, inject=(1,))
    fm = M.factor(A, b, nb, O.CRIT_MAX, 3000.0, tree=O.TREE_BINARY_TT, inject=(1,))
    # the 2^-27 row scaling raises the condition of the remaining system by up to 2^27, so
    # rounding-order differences of later steps grow by that factor (1e-16 -> ~1e-8)
    check_same(fo, fm, tol_margin=1e-5, tol_aug=1e-7)
    assert fm.dec[1] == O.DEC_QR
    forced = np.array([k % 2 for k in range(n)], dtype=np.uint8)
    A2 = A + 8 * np.eye(N)
    fo = O.factor(A2, b, nb, O.CRIT_MAX, 1.0, forced=forced)
    fm = M.factor(A2, b, nb, O.CRIT_MAX, 1.0, forced=forced)
    check_same(fo, fm)
    assert np.array_equal(fm.dec, forced)


def test_float32_storage_matches_numpy_float32():
    A = gauss(256, 5)
    b = A @ np.ones(256)
    fo = O.factor(A, b, 32, O.CRIT_MAX, 2000.0, tree=O.TREE_BINARY_TT, dtype=np.float32)
    fm = M.factor(A, b, 32, O.CRIT_MAX, 2000.0, tree=O.TREE_BINARY_TT, dtype=np.float32)
    assert fm.aug.dtype == np.float32
    # float32 rounding order differs (BLAS vs sequential sums): margins agree to the
    # float32 level amplified by kappa(A_kk)
    check_same(fo, fm, tol_margin=1e-2, tol_aug=1e-4)


def test_force_lu_with_one_tile_is_lapack_gepp():
    A = gauss(40, 0)
    f = M.factor(A, None, 40, O.CRIT_FORCE_LU, 0.0)
    lu, piv = sla.lu_factor(A)
    assert np.allclose(f.U, np.triu(lu), atol=1e-12)


@pytest.mark.parametrize("tree", [O.TREE_FLAT_TS, O.TREE_BINARY_TT, O.TREE_GROUPED])
def test_force_qr_gives_householder_r(tree):
    A = gauss(70, 2)
    f = M.factor(A, None, 16, O.CRIT_FORCE_QR, 0.0, tree=tree, group=3)
    R = f.U
    Rn = np.linalg.qr(A, mode="r")
    sgn = np.sign(np.diag(R)) * np.sign(np.diag(Rn))
    assert np.allclose(R, Rn * sgn[:, None], atol=1e-11 * np.abs(Rn).max())


def test_worst_case_matrix_meets_the_max_test_with_equality():
    n, nb, alpha = 8, 4, 2.0
    A = inputs.worst_case_max(n, nb, alpha).numpy()
    f = M.factor(A, None, nb, O.CRIT_MAX, alpha)
    assert np.all(f.dec == O.DEC_LU)
    assert np.all(f.margin[:-1] == 0.0)            # exact equality at every step but the last
    # growth (1 + alpha)^(n-1) = 3^7 in exact arithmetic: the last tile row of the last
    # tile column ends at 3^7 (every entry of the run is a small dyadic rational)
    assert np.max(np.abs(f.U)) == 3.0 ** 7


@pytest.mark.parametrize("crit", [O.CRIT_MAX, O.CRIT_SUM])
def test_block_diagonally_dominant_is_all_lu(crit):
    A = inputs.block_diag_dominant(6, 8, seed=1).numpy()
    f = M.factor(A, None, 8, crit, 1.0)
    assert np.all(f.dec == O.DEC_LU)


def test_solution_of_ones_system_and_prefix():
    A = inputs.gaussian(512, 7).numpy()
    b = A @ np.ones(512)
    x, f = M.solve(A, b, 64, O.CRIT_MAX, 2000.0, tree=O.TREE_BINARY_TT)
    assert O.backward_error(A, x, b) <= 1e-14
    assert np.max(np.abs(x - 1.0)) <= 1e-9
    g = M.factor(A, b, 64, O.CRIT_MAX, 2000.0, tree=O.TREE_BINARY_TT, steps=3)
    assert g.steps == 3
    assert np.array_equal(g.dec[:3], f.dec[:3]) and np.all(g.dec[3:] == 255)
    assert np.array_equal(g.margin[:3], f.margin[:3])


def test_results_do_not_depend_on_the_thread_count():
    A = gauss(320, 9)
    b = A @ np.ones(320)
    runs = [M.factor(A, b, 32, O.CRIT_MAX, 1500.0, tree=O.TREE_BINARY_TT, threads=t)
            for t in (1, 2, 5)]
    for r in runs[1:]:
        assert np.array_equal(r.aug, runs[0].aug)
        assert np.array_equal(r.margin, runs[0].margin)


def test_errors_match_the_numpy_oracle():
    A = gauss(64, 1)
    A[40, 3] = np.nan
    with pytest.raises(O.NonFinite) as e:
        M.factor(A, None, 16, O.CRIT_MAX, 100.0)
    assert e.value.step == 0
    Z = np.eye(32)
    Z[5, 5] = 0.0
    with pytest.raises(O.Singular) as e:
        M.factor(Z, None, 16, O.CRIT_FORCE_LU, 0.0)
    assert e.value.step == 0 and e.value.row == 5
    f = M.factor(Z, None, 16, O.CRIT_MAX, math.inf)       # zero pivot selects QR
    assert f.dec[0] == O.DEC_QR


@pytest.mark.parametrize("big,small,switch,group", [(2, 1, 8, 4), (1, 2, 5, 3), (2, 0, 20, 8)])
def test_tree_policy_equals_numpy_oracle(big, small, switch, group):
    """The per-step tree policy (small tree below `switch` sub-diagonal tiles) in the C++
    restatement takes the numpy oracle's decisions, margins and final triangle."""
    A = np.random.default_rng(5).standard_normal((640, 640))
    f = O.factor(A, None, 32, O.CRIT_MAX, 2000.0, tree=big, tree_small=small, tree_switch=switch,
                 group=group)
    g = M.factor(A, None, 32, O.CRIT_MAX, 2000.0, tree=big, tree_small=small,
                  tree_switch=switch, group=group, threads=4)
    assert np.array_equal(f.dec, g.dec)
    fin = np.isfinite(f.margin)
    assert np.allclose(f.margin[fin], g.margin[fin], rtol=0, atol=1e-9)
    assert np.allclose(np.triu(g.aug[:, :640]), f.U, rtol=0, atol=1e-10 * np.abs(f.U).max())
