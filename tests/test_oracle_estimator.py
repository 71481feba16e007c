"""Pins of the oracle's Hager-Higham estimate of ||A_kk^-1||_1 (norm_mode = 1), against
facts that do not come from the estimator itself: the exact norm bounds it from above;
it is exact where the maximising vertex is found in one step (entrywise nonnegative
inverse, diagonal and permuted diagonal matrices, 1 x 1); a hand-worked 2 x 2 case; and
the decisions it yields admit LU at least as often as the exact norm."""
import math

import numpy as np
import pytest

from oracle import luqr_oracle as O


def factors(A):
    LU = np.array(A, dtype=np.float64)
    piv, zr = O.getrf(LU)
    assert zr < 0
    return LU, piv


@pytest.mark.parametrize("p", [2, 3, 8, 32, 64])
def test_estimate_is_a_lower_bound(p):
    rng = np.random.default_rng(p)
    for _ in range(40):
        A = rng.standard_normal((p, p))
        LU, piv = factors(A)
        exact = np.max(np.sum(np.abs(np.linalg.inv(A)), axis=0))
        est = O.inv_norm1_est(LU, piv)
        assert est <= exact * (1 + 1e-10)
        assert est > 0.0


def test_one_by_one():
    LU, piv = factors([[-0.25]])
    assert O.inv_norm1_est(LU, piv) == 4.0


@pytest.mark.parametrize("p", [4, 16, 64])
def test_exact_for_nonnegative_inverse(p):
    # M-matrix: positive diagonal, nonpositive off-diagonal, diagonally dominant -> M^-1 >= 0,
    # so sign(A^-1 x) is all ones and the first sub-gradient points at the largest column sum
    rng = np.random.default_rng(p)
    M = -rng.random((p, p)) / p
    np.fill_diagonal(M, 2.0 + rng.random(p))
    assert np.all(np.linalg.inv(M) >= 0)
    LU, piv = factors(M)
    exact = np.max(np.sum(np.abs(np.linalg.inv(M)), axis=0))
    assert abs(O.inv_norm1_est(LU, piv) - exact) <= 1e-12 * exact


@pytest.mark.parametrize("p", [5, 32])
def test_exact_for_signed_permuted_diagonal(p):
    rng = np.random.default_rng(10 + p)
    d = rng.uniform(0.1, 3.0, p) * np.where(rng.random(p) < 0.5, -1.0, 1.0)
    P = np.eye(p)[rng.permutation(p)]
    A = P @ np.diag(d)
    LU, piv = factors(A)
    assert abs(O.inv_norm1_est(LU, piv) - np.max(1.0 / np.abs(d))) <= 1e-14 * np.max(1.0 / np.abs(d))


def test_hand_worked_two_by_two():
    # A = [[4, 1], [2, 3]], A^-1 = [[3, -1], [-2, 4]] / 10, column sums 0.5 and 0.5.
    # x = (1/2, 1/2): A^-1 x = (0.1, 0.1), ||.||_1 = 0.2, xi = (+, +); z = A^-T xi =
    # (0.1, 0.3): j = 1; A^-1 e_1 = (-0.1, 0.4): ||.||_1 = 0.5 > 0.2, sign (-, +) != xi;
    # z = A^-T (-1, 1) = (-0.5, 0.5): |z_0| = |z_1| -> stop at 0.5.  Alternating probe
    # x = (1, -2): A^-1 x = (0.5, -1.0), 2 * 1.5 / 6 = 0.5, not larger.  Estimate 0.5 = exact.
    LU, piv = factors([[4.0, 1.0], [2.0, 3.0]])
    assert abs(O.inv_norm1_est(LU, piv) - 0.5) <= 1e-15


def test_estimate_admits_lu_at_least_as_often():
    rng = np.random.default_rng(3)
    for _ in range(30):
        A = rng.standard_normal((64, 64))
        LU, piv = factors(A)
        below = [float(v) for v in rng.uniform(20.0, 80.0, 3)]
        for alpha in (10.0, 100.0, 1000.0):
            ex = O.decide(O.CRIT_MAX, alpha, LU, piv, -1, below, None, None, norm_mode=0)
            es = O.decide(O.CRIT_MAX, alpha, LU, piv, -1, below, None, None, norm_mode=1)
            assert es.margin >= ex.margin - 1e-12
            if ex.dec == O.DEC_LU:
                assert es.dec == O.DEC_LU


def test_factor_with_estimate_runs_and_solves():
    rng = np.random.default_rng(4)
    N, nb = 256, 32
    A = rng.standard_normal((N, N))
    b = A @ np.ones(N)
    x, f = O.solve(A, b, nb, O.CRIT_MAX, 3000.0, norm_mode=1)
    assert np.all(np.isfinite(x))
    assert O.backward_error(A, x, b) <= 1e-13
    x0, f0 = O.solve(A, b, nb, O.CRIT_MAX, 3000.0)
    # step 0 sees the same tile, so the estimate's margin is at least the exact one
    assert f.margin[0] >= f0.margin[0] - 1e-12
