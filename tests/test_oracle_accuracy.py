"""Pins of the oracle's accuracy measures: the normwise backward error eta and HPL3
(Sec. V-A), on hand-computed cases and through the invariances their definitions imply."""
import numpy as np
import pytest

from oracle import luqr_oracle as O


def test_hand_computed_values():
    A = np.array([[2.0, 0.0], [0.0, 4.0]])
    x = np.array([1.0, 1.0])
    b = np.array([2.0, 5.0])
    # r = b - A x = (0, 1); ||A||_inf = 4, ||x||_inf = 1, ||b||_inf = 5
    assert O.backward_error(A, x, b) == pytest.approx(1.0 / 9.0, rel=1e-15)
    # HPL3 = 1 / (4 * 1 * 2^-53 * 2) = 2^50
    assert O.hpl3(A, x, b) == pytest.approx(2.0 ** 50, rel=1e-15)


def test_exact_solution_gives_zero():
    A = np.array([[1.0, 2.0], [3.0, 4.0]])
    x = np.array([1.0, -1.0])
    b = A @ x
    assert O.backward_error(A, x, b) == 0.0
    assert O.hpl3(A, x, b) == 0.0


def test_scaling_invariances():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((40, 40))
    x = rng.standard_normal(40)
    b = A @ x + 1e-9 * rng.standard_normal(40)
    e, h = O.backward_error(A, x, b), O.hpl3(A, x, b)
    # a common power-of-two scaling of A and b leaves both unchanged (exactly)
    assert O.backward_error(8.0 * A, x, 8.0 * b) == e
    assert O.hpl3(8.0 * A, x, 8.0 * b) == h
    # scaling x and b together rescales eta's numerator and denominator alike
    assert O.backward_error(A, 4.0 * x, 4.0 * b) == pytest.approx(e, rel=1e-12)
    # a permutation of the rows changes nothing
    p = rng.permutation(40)
    assert O.backward_error(A[p], x, b[p]) == pytest.approx(e, rel=1e-14)
