"""The formula-defined special matrices of Table III: each generator against its formula
and a property the formula implies, and the stability pattern of the method on them (the
oracle at N = 64): the Max criterion (alpha = 6000, the paper's special-matrix setting)
is backward stable on every one, while LU restricted to the diagonal tile (FORCE_LU) and
the random choice are not on ris and orthogo."""
import numpy as np
import pytest

from oracle import luqr_oracle as O
from paper_1401_5522_gb300 import inputs


def M(name, N=16, seed=0):
    A = inputs.special(name, N, seed)
    assert A.stride() == (1, N)
    return A.numpy()


def test_hilbert_inverse_is_the_classic_integer_matrix():
    H = M("hilb", 4)
    assert H[2, 3] == 1.0 / 6.0
    inv = np.array([[16, -120, 240, -140], [-120, 1200, -2700, 1680],
                    [240, -2700, 6480, -4200], [-140, 1680, -4200, 2800]], dtype=float)
    assert np.allclose(np.linalg.inv(H), inv, rtol=1e-9, atol=0)


def test_lehmer_formula_and_tridiagonal_inverse():
    A = M("lehmer", 12)
    assert A[1, 5] == 2.0 / 6.0 and np.array_equal(A, A.T)
    inv = np.linalg.inv(A)
    off = np.abs(np.triu(inv, 2))
    assert off.max() <= 1e-9 * np.abs(inv).max()
    assert np.all(np.linalg.eigvalsh(A) > 0)


def test_orthogo_is_symmetric_orthogonal():
    A = M("orthogo", 20)
    assert np.array_equal(A, A.T)
    assert np.allclose(A.T @ A, np.eye(20), atol=1e-13)
    assert A[0, 0] == pytest.approx(np.sqrt(2 / 21) * np.sin(np.pi / 21), rel=1e-15)


def test_house_reflects_its_vector():
    A = M("house", 10, seed=3)
    assert np.allclose(A @ A, np.eye(10), atol=1e-14) and np.allclose(A, A.T, atol=0)
    assert np.isclose(np.linalg.det(A), -1.0)


def test_parter_toeplitz_with_singular_values_near_pi():
    A = M("parter", 64)
    assert np.array_equal(A[1:, 1:], A[:-1, :-1])
    assert A[3, 1] == 1.0 / 2.5
    sv = np.linalg.svd(A, compute_uv=False)
    assert np.median(np.abs(sv - np.pi)) < 1e-2


def test_ris_hankel_with_eigenvalues_near_half_pi():
    A = M("ris", 64)
    assert np.array_equal(A[1:, :-1], A[:-1, 1:])          # depends on i + j only
    assert A[0, 0] == 0.5 / (64 - 2 + 1.5)
    ev = np.linalg.eigvalsh(A)
    assert np.median(np.abs(np.abs(ev) - np.pi / 2)) < 1e-2


def test_demmel_row_scaling():
    N = 32
    A = M("demmel", N, seed=5)
    d = 10.0 ** (14.0 * np.arange(N) / N)
    E = A / d.reshape(-1, 1) - np.eye(N)
    assert E.min() >= 0.0 and E.max() <= 1e-7 * (1 + 1e-12)


STABLE_BAR = 1e-14


@pytest.mark.parametrize("name", inputs.SPECIAL)
def test_max_criterion_is_stable_on_every_special_matrix(name):
    N, nb = 64, 16
    A = M(name, N, seed=1)
    b = A @ np.ones(N)
    x, f = O.solve(A, b, nb, O.CRIT_MAX, 6000.0)
    assert O.backward_error(A, x, b) <= STABLE_BAR


@pytest.mark.parametrize("name", ["ris", "orthogo"])
def test_tile_restricted_lu_and_random_choice_fail_where_max_does_not(name):
    N, nb = 64, 16
    A = M(name, N, seed=1)
    b = A @ np.ones(N)
    x, _ = O.solve(A, b, nb, O.CRIT_FORCE_LU, 0.0)
    assert O.backward_error(A, x, b) > 1e-3
    x, f = O.solve(A, b, nb, O.CRIT_RANDOM, 50.0, seed=0)
    assert O.backward_error(A, x, b) > 1e-3 and np.any(f.dec == O.DEC_LU)
