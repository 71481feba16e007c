"""Pins of the diagonal-domain variant of the Factor step (Sec. II-B: pivoting across the
tiles of the diagonal domain instead of inside the diagonal tile only)."""
import numpy as np
import pytest

from oracle import luqr_oracle as O


def gauss(N, seed):
    return np.random.default_rng(seed).standard_normal((N, N))


@pytest.mark.parametrize("N,nb", [(96, 32), (100, 16)])
def test_all_lu_over_the_whole_panel_is_lapack_gepp(N, nb):
    """FORCE_LU with a domain spanning every remaining tile is Gaussian elimination with
    partial pivoting: same pivot rows as LAPACK dgetrf and the same U."""
    la = pytest.importorskip("scipy.linalg")
    A = gauss(N, 3)
    f = O.factor(A, None, nb, O.CRIT_FORCE_LU, 0.0, domain=10 ** 6)
    lu, ipiv = la.lu_factor(A)
    n = f.n
    ours = []
    for k in range(n):
        r0, r1 = O.tile_bounds(k, nb, N)
        dd, dpiv = f.domain_piv.get(k, (1, f.piv[k]))
        ours.extend(int(r0 + p) for p in dpiv[:r1 - r0])
    assert ours == [int(p) for p in ipiv]
    assert np.max(np.abs(f.U - np.triu(lu))) <= 1e-12 * np.max(np.abs(lu))


def test_domain_one_is_the_tile_variant():
    A = gauss(128, 4)
    b = A @ np.ones(128)
    f1 = O.factor(A, b, 32, O.CRIT_MAX, 3000.0, domain=1)
    f0 = O.factor(A, b, 32, O.CRIT_MAX, 3000.0)
    assert np.array_equal(f1.dec, f0.dec) and np.array_equal(f1.aug, f0.aug)


def test_domain_admits_more_lu_steps():
    """Pivoting over the domain raises the smallest singular value of the factored tile,
    so the criterion passes at least as often (summed over random matrices)."""
    lu1 = lu4 = 0
    for seed in range(8):
        A = gauss(256, 100 + seed)
        lu1 += int(np.sum(O.factor(A, None, 32, O.CRIT_MAX, 3000.0).dec == O.DEC_LU))
        lu4 += int(np.sum(O.factor(A, None, 32, O.CRIT_MAX, 3000.0, domain=4).dec == O.DEC_LU))
    assert lu4 > lu1


@pytest.mark.parametrize("crit,alpha", [(O.CRIT_MAX, 3000.0), (O.CRIT_SUM, 20000.0),
                                        (O.CRIT_FORCE_LU, 0.0)])
def test_domain_runs_solve_and_replay(crit, alpha):
    N = 256
    A = gauss(N, 7)
    b = A @ np.ones(N)
    x, f = O.solve(A, b, 32, crit, alpha, domain=3)
    assert O.backward_error(A, x, b) <= 1e-13
    assert any(k in f.domain_piv for k in range(f.n))
    b2 = np.random.default_rng(8).standard_normal(N)
    x2 = O.replay_solve(f, b2)
    assert O.backward_error(A, x2, b2) <= 1e-13


def test_domain_with_mumps_and_float32_emulation():
    A = gauss(192, 9)
    b = A @ np.ones(192)
    x, f = O.solve(A, b, 32, O.CRIT_MUMPS, 2.1, domain=2)
    assert O.backward_error(A, x, b) <= 1e-13
    x32, f32 = O.solve(A, b, 32, O.CRIT_MAX, 3000.0, domain=2, dtype=np.float32)
    assert O.backward_error(A, x32.astype(np.float64), b) <= 1e-4
    assert f32.aug.dtype == np.float32
