"""Pins of the oracle's step loop (Alg. 1-4), criteria (Eq. 2-4) and solve (Sec. II-D).

References used: LAPACK GEPP (scipy), numpy's QR, a scalar Gaussian elimination with
tile-restricted pivoting written below, the growth example and bounds of Sec. III,
block diagonal dominance (Sec. III-B), hand-worked 2x2-tile examples, Table I/II.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import luqr_oracle as O
from paper_1401_5522_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def gauss(N, seed):
    return np.random.default_rng(seed).standard_normal((N, N))


# ----------------------------------------------------------------- limits of alpha
def test_force_lu_with_one_tile_is_lapack_gepp():
    A = gauss(24, 0)
    b = A @ np.ones(24)
    f = O.factor(A, b, 24, O.CRIT_FORCE_LU, 0.0)
    lu, piv = sla.lu_factor(A)
    assert np.allclose(np.triu(f.aug[:, :24]), np.triu(lu), atol=1e-12)


def scalar_ge_tile_pivoting(A, nb):
    """Brute force: scalar Gaussian elimination whose pivot search at column c is
    restricted to rows c .. end of c's diagonal tile; every row below c is eliminated."""
    U = A.astype(np.float64).copy()
    N = U.shape[0]
    for c in range(N):
        end = min((c // nb + 1) * nb, N)
        p = c + int(np.argmax(np.abs(U[c:end, c])))
        U[[c, p], c:] = U[[p, c], c:]
        for r in range(c + 1, N):
            f = U[r, c] / U[c, c]
            U[r, c:] -= f * U[c, c:]
    return np.triu(U)


@pytest.mark.parametrize("N,nb", [(32, 8), (30, 8), (20, 5)])
def test_force_lu_is_block_lu_with_tile_pivoting(N, nb):
    A = gauss(N, 1) + 4 * np.eye(N)
    f = O.factor(A, None, nb, O.CRIT_FORCE_LU, 0.0)
    ref = scalar_ge_tile_pivoting(A, nb)
    assert np.allclose(f.U, ref, atol=1e-10 * np.abs(ref).max())
    # alpha = +inf behaves as FORCE_LU for the Max criterion
    g = O.factor(A, None, nb, O.CRIT_MAX, math.inf)
    assert np.all(g.dec == O.DEC_LU)
    assert np.array_equal(g.aug, f.aug)


@pytest.mark.parametrize("tree", [O.TREE_FLAT_TS, O.TREE_BINARY_TT, O.TREE_GROUPED])
@pytest.mark.parametrize("N,nb", [(40, 8), (37, 8), (64, 16)])
def test_force_qr_gives_householder_r(tree, N, nb):
    A = gauss(N, 2)
    f = O.factor(A, None, nb, O.CRIT_FORCE_QR, 0.0, tree=tree, group=3)
    R = f.U
    Rn = np.linalg.qr(A, mode="r")
    sgn = np.sign(np.diag(R)) * np.sign(np.diag(Rn))
    assert np.allclose(R, Rn * sgn[:, None], atol=1e-11 * np.abs(Rn).max())
    # alpha = 0 is the same run for every criterion
    for crit in (O.CRIT_MAX, O.CRIT_SUM, O.CRIT_MUMPS):
        g = O.factor(A, None, nb, crit, 0.0, tree=tree, group=3)
        assert np.all(g.dec == O.DEC_QR)
        assert np.array_equal(g.aug, f.aug)


# ----------------------------------------------------------------- solve
@pytest.mark.parametrize("crit,alpha", [(O.CRIT_MAX, 100.0), (O.CRIT_MAX, 3000.0),
                                        (O.CRIT_SUM, 1e4), (O.CRIT_MUMPS, 2.1),
                                        (O.CRIT_FORCE_LU, 0.0), (O.CRIT_FORCE_QR, 0.0)])
@pytest.mark.parametrize("tree", [O.TREE_FLAT_TS, O.TREE_BINARY_TT])
def test_solution_of_ones_system(crit, alpha, tree):
    N, nb = 72, 16
    A = gauss(N, 3)
    b = A @ np.ones(N)
    x, f = O.solve(A, b, nb, crit, alpha, tree=tree)
    assert O.backward_error(A, x, b) < 1e-13
    assert np.max(np.abs(x - 1.0)) < 1e-8
    # second pass on the same b reproduces the augmented solution
    x2 = O.replay_solve(f, b)
    assert np.allclose(x, x2, rtol=0, atol=1e-12)


def test_mixed_sequence_appears_at_paper_scale_alpha():
    N, nb = 256, 32
    A = gauss(N, 4)
    f = O.factor(A, None, nb, O.CRIT_MAX, 3000.0)
    assert 0 < int(np.sum(f.dec)) < f.n


def test_ragged_native_equals_identity_padding():
    N, nb = 45, 8
    n = 6
    A = gauss(N, 5)
    b = A @ np.ones(N)
    Np = n * nb
    Ap = np.eye(Np)
    Ap[:N, :N] = A
    bp = np.zeros(Np)
    bp[:N] = b
    for crit, alpha in [(O.CRIT_MAX, 50.0), (O.CRIT_MAX, 1e5), (O.CRIT_MUMPS, 2.0)]:
        for tree in (O.TREE_FLAT_TS, O.TREE_BINARY_TT):
            x, f = O.solve(A, b, nb, crit, alpha, tree=tree)
            xp, fp = O.solve(Ap, bp, nb, crit, alpha, tree=tree)
            assert np.array_equal(f.dec[:-1], fp.dec[:-1])
            assert np.allclose(x, xp[:N], atol=1e-12)
            assert np.allclose(xp[N:], 0.0)
            assert np.allclose(f.U, fp.U[:N, :N], atol=1e-12)


def test_runtime_injection_forces_qr_and_keeps_solution():
    N, nb = 64, 8
    A = gauss(N, 6) + 10 * np.eye(N)
    b = A @ np.ones(N)
    x0, f0 = O.solve(A, b, nb, O.CRIT_MAX, 1e6)
    inj = [2]
    x1, f1 = O.solve(A, b, nb, O.CRIT_MAX, 1e6, inject=inj)
    assert all(f1.dec[k] == O.DEC_QR for k in inj)
    assert np.all(f1.dec[:inj[0]] == f0.dec[:inj[0]])
    # the scaling is an exact equivalence transform, but it raises the condition
    # number of the remaining system by up to 2^27, so x keeps ~1e-7 forward error
    assert np.allclose(x1, 1.0, atol=1e-5)
    assert np.allclose(O.replay_solve(f1, b), x1, atol=1e-12)


def test_nonfinite_panel_raises():
    A = gauss(16, 7)
    A[9, 3] = np.nan
    with pytest.raises(O.NonFinite) as e:
        O.factor(A, None, 8, O.CRIT_MAX, 10.0)
    assert e.value.step == 0


def test_force_lu_zero_pivot_raises_singular():
    A = gauss(16, 8)
    A[0:8, 0:8] = 0.0
    with pytest.raises(O.Singular):
        O.factor(A, None, 8, O.CRIT_FORCE_LU, 0.0)
    f = O.factor(A, None, 8, O.CRIT_MAX, 1e9)
    assert f.dec[0] == O.DEC_QR


def test_float32_factorization_emulation_is_single_precision_accurate():
    N, nb = 64, 16
    A = gauss(N, 9)
    b = A @ np.ones(N)
    x, f = O.solve(A, b, nb, O.CRIT_MAX, 100.0, dtype=np.float32)
    assert f.aug.dtype == np.float32
    eta = O.backward_error(A, x, b)
    assert 1e-10 < eta < 1e-5


# ----------------------------------------------------------------- Sec. III pins
def test_worst_case_max_matrix_equality_and_growth():
    n, nb, alpha = 8, 4, 2.0
    A = inputs.worst_case_max(n, nb, alpha).numpy()
    f = O.factor(A, None, nb, O.CRIT_MAX, alpha, track_growth=True)
    assert np.all(f.dec == O.DEC_LU)
    assert np.all(f.margin[:-1] == 0.0)                     # Eq. 2 holds with equality
    assert np.all(f.lhs[:-1] == f.rhs[:-1])
    growth = max(f.growth) / f.growth[0]
    assert growth == (1.0 + alpha) ** (n - 1)               # 3^7 = 2187 exactly
    # Sum criterion with the same alpha rejects the first panel (n-1 > 1 tiles below)
    g = O.factor(A, None, nb, O.CRIT_SUM, alpha)
    assert g.dec[0] == O.DEC_QR


@pytest.mark.parametrize("crit", [O.CRIT_MAX, O.CRIT_SUM])
def test_block_diagonally_dominant_is_all_lu(crit):
    n, nb = 6, 5
    A = inputs.block_diag_dominant(n, nb, seed=3).numpy()
    f = O.factor(A, None, nb, crit, 1.0, track_growth=True)
    assert np.all(f.dec == O.DEC_LU)
    if crit == O.CRIT_SUM:
        assert max(f.growth) / f.growth[0] <= n * (1 + 1e-12)


@pytest.mark.parametrize("crit,alpha", [(O.CRIT_MAX, 1500.0), (O.CRIT_SUM, 8000.0)])
def test_growth_bounds_hold_at_every_lu_step(crit, alpha):
    N, nb = 96, 8
    n = N // nb
    A = gauss(N, 11)
    snaps = {}

    def hook(k, aug, fact):
        snaps[k] = aug[:, :N].copy()

    f = O.factor(A, None, nb, crit, alpha, on_step=hook)
    tn = lambda M, i, j: O.norm1(M[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb])
    checked = 0
    for k in range(n - 1):
        if f.dec[k] != O.DEC_LU:
            continue
        before, after = snaps[k], snaps[k + 1]
        for j in range(k + 1, n):
            akj = tn(before, k, j)
            if crit == O.CRIT_MAX:
                for i in range(k + 1, n):
                    assert tn(after, i, j) <= (tn(before, i, j) + alpha * akj) * (1 + 1e-12)
            else:
                lhs = sum(tn(after, i, j) for i in range(k + 1, n))
                rhs = sum(tn(before, i, j) for i in range(k + 1, n)) + alpha * akj
                assert lhs <= rhs * (1 + 1e-12)
            checked += 1
    assert checked > 0


# ----------------------------------------------------------------- hand-worked decisions
def test_max_and_sum_margins_two_by_two_tiles():
    # A_11 = diag(2, 4)   -> ||A_11^-1||_1 = 1/2, lhs = alpha * 2
    # A_21 = [[1, 0], [3, 1]] -> ||A_21||_1 = 4 ; only one tile below, so Max = Sum = 4
    A = np.array([[2.0, 0.0, 1.0, 0.0],
                  [0.0, 4.0, 0.0, 1.0],
                  [1.0, 0.0, 5.0, 0.0],
                  [3.0, 1.0, 0.0, 5.0]])
    f = O.factor(A, None, 2, O.CRIT_MAX, 2.0)
    assert f.dec[0] == O.DEC_LU and f.lhs[0] == 4.0 and f.rhs[0] == 4.0 and f.margin[0] == 0.0
    f = O.factor(A, None, 2, O.CRIT_MAX, 1.0)
    assert f.dec[0] == O.DEC_QR and f.margin[0] == -1.0
    f = O.factor(A, None, 2, O.CRIT_SUM, 8.0)
    assert f.dec[0] == O.DEC_LU and f.margin[0] == 2.0


def test_mumps_two_by_two_tiles_by_hand():
    # A_11 = [[1, 2], [4, 1]]: local_max = (4, 2); GETRF pivots row 2 -> U = [[4, 1], [0, 1.75]]
    # pivot = (4, 1.75); growth g = (4/4, 1.75/2) = (1, 0.875)
    # A_21 = [[8, 0], [1, 3]]: away_max = (8, 3)
    # R2 reading: est(j) = away(j) * g(j) = (8, 2.625); LU iff alpha*pivot(j) >= est(j)
    #   j=0: 4 alpha >= 8 -> alpha >= 2 ; j=1: 1.75 alpha >= 2.625 -> alpha >= 1.5
    A = np.array([[1.0, 2.0, 1.0, 0.0],
                  [4.0, 1.0, 0.0, 1.0],
                  [8.0, 0.0, 9.0, 0.0],
                  [1.0, 3.0, 0.0, 9.0]])
    assert O.factor(A, None, 2, O.CRIT_MUMPS, 2.0).dec[0] == O.DEC_LU
    f = O.factor(A, None, 2, O.CRIT_MUMPS, 1.9)
    assert f.dec[0] == O.DEC_QR
    assert abs(f.margin[0] - math.log2(1.9 * 4 / 8)) < 1e-15
    # R1 reading: est = away(j) * prod_{l<j} g(l) = (8, 3 * 1) ; j=1: 1.75 alpha >= 3
    assert O.factor(A, None, 2, O.CRIT_MUMPS, 1.7, mumps_mode=1).dec[0] == O.DEC_QR
    assert O.factor(A, None, 2, O.CRIT_MUMPS, 2.0, mumps_mode=1).dec[0] == O.DEC_LU


def test_last_step_is_lu_iff_nonsingular():
    A = gauss(16, 12)
    f = O.factor(A, None, 8, O.CRIT_MAX, 1e-3)
    assert f.dec[-1] == O.DEC_LU
    f = O.factor(A, None, 8, O.CRIT_MAX, 0.0)
    assert f.dec[-1] == O.DEC_QR


# ----------------------------------------------------------------- elimination trees
def test_elimination_lists():
    E = O.elimination_ops
    assert E(0, 4, O.TREE_FLAT_TS) == [("geqrt", 0), ("ts", 1, 0), ("ts", 2, 0), ("ts", 3, 0)]
    assert E(1, 6, O.TREE_BINARY_TT) == [("geqrt", 1), ("geqrt", 2), ("geqrt", 3), ("geqrt", 4),
                                         ("geqrt", 5), ("tt", 2, 1), ("tt", 4, 3), ("tt", 3, 1),
                                         ("tt", 5, 1)]
    assert E(0, 7, O.TREE_GROUPED, group=3) == [("geqrt", 0), ("ts", 1, 0), ("ts", 2, 0),
                                                ("geqrt", 3), ("ts", 4, 3), ("ts", 5, 3),
                                                ("geqrt", 6), ("tt", 3, 0), ("tt", 6, 0)]
    # every tile below the diagonal is eliminated exactly once
    for tree in (O.TREE_FLAT_TS, O.TREE_BINARY_TT, O.TREE_GROUPED):
        for n in range(1, 12):
            ops = E(0, n, tree, group=3)
            killed = sorted(op[1] for op in ops if op[0] != "geqrt")
            assert killed == list(range(1, n))


# ----------------------------------------------------------------- Table I / Table II
def test_flop_counter_matches_table1_closed_form():
    n, nb = 10, 4
    N = n * nb
    A = gauss(N, 13)
    f_lu = O.factor(A, None, nb, O.CRIT_FORCE_LU, 0.0)
    f_qr = O.factor(A, None, nb, O.CRIT_FORCE_QR, 0.0)
    lu_units = sum(2 / 3 + 2 * m + 2 * m * m for m in range(n))
    qr_units = sum(4 / 3 + 4 * m + 4 * m * m for m in range(n))
    assert math.isclose(f_lu.flops, lu_units * nb ** 3)
    assert math.isclose(f_qr.flops, qr_units * nb ** 3)
    assert math.isclose(f_qr.flops, 2 * f_lu.flops)
    # leading term (2/3) n^3 nb^3 = (2/3) N^3
    assert abs(f_lu.flops / ((2 / 3) * N ** 3) - 1) < 3.5 / n


def test_table2_metric_arithmetic():
    rows = []
    with open(os.path.join(HERE, "golden", "table2_n20000.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, alpha, t, plu, fake, true, fpk, tpk = line.split()
            rows.append((name, float(t), float(plu), float(fake), float(true), float(fpk),
                         float(tpk)))
    N, peak = 20000, 1091.0
    for name, t, plu, fake, true, fpk, tpk in rows:
        assert abs(O.normalized_gflops(N, t) / fake - 1) < 3e-3, name
        if name.startswith("LUQR") or name == "HQR":
            assert abs(O.true_gflops(N, t, plu / 100.0) / true - 1) < 3e-3, name
        assert abs(100 * fake / peak - fpk) < 0.1, name   # printed to 0.1%


def _mumps_case(seed, p=16):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((p, p))
    local = np.max(np.abs(A), axis=0)
    away = rng.uniform(0.2, 3.0, p) * local          # column maxima of the tiles below
    LU = A.copy()
    piv, zr = O.getrf(LU)
    assert zr < 0
    return LU, piv, local, away


@pytest.mark.parametrize("seed", range(6))
def test_mumps_default_reading_closed_form(seed):
    """Default reading: est(j) = away(j) pivot(j) / local(j) and LU iff alpha pivot(j) >=
    est(j) for every j, i.e. LU iff alpha >= max_j away(j) / local(j), with margin
    min_j log2(alpha local(j) / away(j)).  Alphas sit between the sorted thresholds."""
    LU, piv, local, away = _mumps_case(seed)
    thr = np.sort(away / local)
    for a in np.concatenate([[thr[0] / 2], np.sqrt(thr[:-1] * thr[1:]), [thr[-1] * 2]]):
        sd = O.decide(O.CRIT_MUMPS, float(a), LU, piv, -1, [1.0], local, away, mumps_mode=0)
        assert sd.dec == (O.DEC_LU if a >= thr[-1] else O.DEC_QR)
        assert sd.margin == pytest.approx(float(np.min(np.log2(a * local / away))), abs=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_mumps_cumulative_reading_closed_form(seed):
    """Cumulative reading: est(j) = away(j) prod_{l<j} pivot(l)/local(l).  In logs, LU iff
    log alpha >= max_j [log away(j) + sum_{l<j} (log pivot(l) - log local(l)) - log pivot(j)]
    (prefix sums computed independently of the oracle's running product)."""
    LU, piv, local, away = _mumps_case(100 + seed)
    lp = np.log(np.abs(np.diag(LU)))
    prefix = np.concatenate([[0.0], np.cumsum(lp - np.log(local))[:-1]])
    t = np.log(away) + prefix - lp
    tmax = float(np.max(t))
    for a in (np.exp(tmax - 1.0), np.exp(tmax + 1.0), np.exp(tmax - 0.01), np.exp(tmax + 0.01)):
        sd = O.decide(O.CRIT_MUMPS, float(a), LU, piv, -1, [1.0], local, away, mumps_mode=1)
        assert sd.dec == (O.DEC_LU if np.log(a) >= tmax else O.DEC_QR)
        assert sd.margin == pytest.approx(float(np.min(np.log(a) - t)) / np.log(2.0), abs=1e-9)


@pytest.mark.parametrize("big,small,switch", [(O.TREE_BINARY_TT, O.TREE_FLAT_TS, 8),
                                              (O.TREE_GROUPED, O.TREE_BINARY_TT, 5),
                                              (O.TREE_FLAT_TS, O.TREE_BINARY_TT, 20)])
def test_per_step_tree_policy(big, small, switch):
    """A tree that changes with the step is still Householder QR on FORCE_QR (R equal to
    numpy's up to row signs); switch 0 is the big tree and a switch above n the small tree,
    step for step (bitwise)."""
    A = gauss(400, 2)
    f = O.factor(A, None, 16, O.CRIT_FORCE_QR, 0.0, tree=big, tree_small=small,
                 tree_switch=switch, group=3)
    Rn = np.linalg.qr(A, mode="r")
    sgn = np.sign(np.diag(f.U)) * np.sign(np.diag(Rn))
    assert np.allclose(f.U, Rn * sgn[:, None], atol=1e-11 * np.abs(Rn).max())
    g0 = O.factor(A, None, 16, O.CRIT_MAX, 2000.0, tree=big, tree_small=small, tree_switch=0,
                  group=3)
    g1 = O.factor(A, None, 16, O.CRIT_MAX, 2000.0, tree=big, group=3)
    assert np.array_equal(g0.aug, g1.aug)
    h0 = O.factor(A, None, 16, O.CRIT_MAX, 2000.0, tree=big, tree_small=small, tree_switch=99,
                  group=3)
    h1 = O.factor(A, None, 16, O.CRIT_MAX, 2000.0, tree=small, group=3)
    assert np.array_equal(h0.aug, h1.aug) and np.array_equal(h0.dec, h1.dec)
