"""Pins of LU variant A2 (Sec. II-B: the diagonal tile factored by QR; Eliminate A_ik U^-1,
Apply Q^T A_kj, Update as in A1).  Both variants form the same Schur complement
A_ij - A_ik A_kk^-1 A_kj, so with an exact inverse norm they take the same decisions and
reach the same solution; only row k of the triangle differs."""
import numpy as np
import pytest

from oracle import luqr_oracle as O


def gauss(N, seed):
    return np.random.default_rng(seed).standard_normal((N, N))


def test_inverse_norm_from_qr_factors():
    rng = np.random.default_rng(0)
    for p in (1, 5, 32):
        A = rng.standard_normal((p, p))
        QR = A.copy()
        tau = O.geqrt(QR)
        exact = np.max(np.sum(np.abs(np.linalg.inv(A)), axis=0))
        assert O.inv_norm1_qr(QR, tau) == pytest.approx(exact, rel=1e-10)


def test_single_tile_is_a_qr_solve():
    A = gauss(48, 1)
    b = A @ np.ones(48)
    x, f = O.solve(A, b, 48, O.CRIT_FORCE_LU, 0.0, lu_variant="A2")
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-12)
    Q, R = np.linalg.qr(A)
    assert np.allclose(np.abs(np.diag(f.U)), np.abs(np.diag(R)), rtol=1e-12)


@pytest.mark.parametrize("crit,alpha", [(O.CRIT_MAX, 3000.0), (O.CRIT_SUM, 20000.0),
                                        (O.CRIT_FORCE_LU, 0.0)])
def test_same_decisions_and_solution_as_a1(crit, alpha):
    N, nb = 256, 32
    A = gauss(N, 2)
    b = A @ np.ones(N)
    x1, f1 = O.solve(A, b, nb, crit, alpha, lu_variant="A1")
    x2, f2 = O.solve(A, b, nb, crit, alpha, lu_variant="A2")
    assert np.array_equal(f1.dec, f2.dec)
    assert crit == O.CRIT_FORCE_LU or set(f1.dec.tolist()) == {0, 1}
    fin = np.isfinite(f1.margin)
    assert np.all(np.abs(f1.margin[fin] - f2.margin[fin]) <= 1e-9)
    assert np.max(np.abs(x1 - x2)) <= 1e-10
    assert O.backward_error(A, x2, b) <= 1e-13
    y = O.replay_solve(f2, b)
    assert np.max(np.abs(y - x2)) <= 1e-10


def test_schur_complement_after_an_lu_step_matches_a1():
    N, nb = 128, 32
    A = gauss(N, 3)
    seen = {}

    def hook(tag):
        def f(k, aug, fact):
            if k == 1:
                seen[tag] = aug[nb:, nb:N].copy()
        return f

    O.factor(A, None, nb, O.CRIT_FORCE_LU, 0.0, lu_variant="A1", on_step=hook("A1"))
    O.factor(A, None, nb, O.CRIT_FORCE_LU, 0.0, lu_variant="A2", on_step=hook("A2"))
    assert np.max(np.abs(seen["A1"] - seen["A2"])) <= 1e-12 * np.max(np.abs(seen["A1"]))
