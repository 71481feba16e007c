"""Pins of the oracle's tile kernels against LAPACK and textbook definitions.

Nothing here compares the oracle with itself: each reference is a LAPACK routine
(through scipy), a closed form, or an explicit matrix product built in the test.
"""
import numpy as np
import pytest
import scipy.linalg as sla
from scipy.linalg import lapack

from oracle import luqr_oracle as O

RNG = np.random.default_rng(1234)


def rand(p, q=None):
    return RNG.standard_normal((p, p if q is None else q))


@pytest.mark.parametrize("p", [1, 2, 5, 16, 33])
def test_getrf_matches_lapack_dgetrf(p):
    A = rand(p)
    T = A.copy()
    piv, zero_row = O.getrf(T)
    lu, lpiv = sla.lu_factor(A)
    assert zero_row == -1
    assert np.array_equal(piv, lpiv)          # identical pivot sequence (first max index)
    assert np.allclose(T, lu, rtol=0, atol=1e-13 * np.abs(lu).max())


def test_getrf_tie_takes_first_row():
    A = np.array([[1.0, 2.0, 0.0], [-3.0, 1.0, 1.0], [3.0, 0.5, 2.0]])
    T = A.copy()
    piv, _ = O.getrf(T)
    assert piv[0] == 1            # |-3| and |3| tie: the first row wins


def test_getrf_zero_pivot_reported():
    A = np.array([[0.0, 1.0], [0.0, 2.0]])
    T = A.copy()
    _, zero_row = O.getrf(T)
    assert zero_row == 0


@pytest.mark.parametrize("shape", [(8, 8), (12, 5), (5, 12), (1, 4), (4, 1)])
def test_geqrt_matches_lapack_dgeqrf(shape):
    A = rand(*shape)
    T = A.copy()
    tau = O.geqrt(T)
    qr, ltau, work, info = lapack.dgeqrf(A)
    assert info == 0
    # same reflector convention: R, V and tau agree to rounding
    assert np.allclose(tau, ltau[:len(tau)], rtol=0, atol=1e-13)
    assert np.allclose(T, qr, rtol=0, atol=1e-12 * np.abs(qr).max())


def test_unmqr_matches_lapack_dormqr():
    A = rand(10)
    C = rand(10, 7)
    T = A.copy()
    tau = O.geqrt(T)
    C1 = C.copy()
    O.unmqr(T, tau, C1)
    qr, ltau, _, _ = lapack.dgeqrf(A)
    ref, _, info = lapack.dormqr("L", "T", qr, ltau, C, lwork=100)
    assert info == 0
    assert np.allclose(C1, ref, atol=1e-13)


def _explicit_q_pair(apply_fn, V, tau, p1, p2):
    """Q^T of a pair kernel as an explicit (p1+p2) x (p1+p2) matrix, by applying it to I."""
    I = np.eye(p1 + p2)
    C1 = I[:p1].copy()
    C2 = I[p1:].copy()
    apply_fn(V, tau, C1, C2)
    return np.vstack([C1, C2])


@pytest.mark.parametrize("q,p", [(6, 6), (6, 3), (1, 1)])
def test_tsqrt_is_qr_of_stacked(q, p):
    R0 = np.triu(rand(q))
    A0 = rand(p, q)
    R = R0.copy()
    A = A0.copy()
    tau = O.tsqrt(R, A)
    QT = _explicit_q_pair(O.tsmqr, A, tau, q, p)
    S = np.vstack([R0, A0])
    assert np.allclose(QT @ QT.T, np.eye(p + q), atol=1e-13)
    out = QT @ S
    assert np.allclose(out[:q], np.triu(R), atol=1e-12)
    assert np.allclose(out[q:], 0.0, atol=1e-12)
    # R agrees with numpy's QR of the stacked matrix up to row signs
    Rn = np.linalg.qr(S, mode="r")
    assert np.allclose(np.abs(np.triu(R)), np.abs(Rn[:q]), atol=1e-12)


@pytest.mark.parametrize("q,p", [(6, 6), (6, 4), (3, 1)])
def test_ttqrt_is_qr_of_two_triangles(q, p):
    R0 = np.triu(rand(q))
    B0 = np.triu(rand(p, q))
    R = R0.copy()
    B = B0.copy()
    tau = O.ttqrt(R, B)
    assert np.allclose(np.tril(B, -1), 0.0)          # reflector tails stay upper triangular
    QT = _explicit_q_pair(O.ttmqr, B, tau, q, p)
    S = np.vstack([R0, B0])
    assert np.allclose(QT @ QT.T, np.eye(p + q), atol=1e-13)
    out = QT @ S
    assert np.allclose(out[:q], np.triu(R), atol=1e-12)
    assert np.allclose(out[q:], 0.0, atol=1e-12)
    # on a triangular input the square (TS) kernel computes the same thing
    R2 = R0.copy()
    B2 = B0.copy()
    tau2 = O.tsqrt(R2, B2)
    assert np.array_equal(tau, tau2)
    assert np.array_equal(R, R2)
    assert np.array_equal(B, B2)


@pytest.mark.parametrize("p", [1, 3, 17])
def test_inverse_norm_matches_explicit_inverse(p):
    A = rand(p) + 0.1 * np.eye(p)
    T = A.copy()
    piv, _ = O.getrf(T)
    got = O.inv_norm1(T, piv)
    ref = np.linalg.norm(np.linalg.inv(A), 1)
    assert abs(got - ref) <= 1e-12 * ref


def test_trsm_and_swptrsm_match_triangular_solves():
    A = rand(9)
    T = A.copy()
    piv, _ = O.getrf(T)
    L = np.tril(T, -1) + np.eye(9)
    U = np.triu(T)
    X = rand(5, 9)
    X1 = X.copy()
    O.trsm_right_upper(X1, T)
    assert np.allclose(X1 @ U, X, atol=1e-12)
    C = rand(9, 4)
    C1 = C.copy()
    O.swptrsm(C1, T, piv)
    P = np.eye(9)
    O.apply_row_swaps(P, piv)
    assert np.allclose(L @ C1, P @ C, atol=1e-12)
    # P A = L U
    assert np.allclose(P @ A, L @ U, atol=1e-12)


def test_householder_zero_tail_is_identity():
    beta, tau, v = O.householder(-2.5, np.zeros(3))
    assert tau == 0.0 and beta == -2.5 and np.all(v == 0.0)


def test_householder_sign_of_zero_head():
    beta, tau, v = O.householder(0.0, np.array([3.0, 4.0]))
    assert beta == -5.0 and tau == 1.0
    assert np.allclose(v, [0.6, 0.8])


def test_norm1_is_max_column_sum():
    T = np.array([[1.0, -4.0], [-2.0, 1.0], [3.0, 0.5]])
    assert O.norm1(T) == 6.0
