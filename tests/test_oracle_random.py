"""Pins of the random-choice criterion (Sec. V-B, Fig. 2 fourth row: LU with probability
alpha/100 at each step) and of the SplitMix64 draws both sides use."""
import numpy as np
import pytest

from oracle import luqr_oracle as O


def test_splitmix64_reference_outputs():
    # first three outputs of the published SplitMix64 generator with state 0
    assert [O.splitmix64_at(0, i) for i in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_draws_are_uniform_53_bit():
    u = np.array([O.random_draw(12345, k) for k in range(4000)])
    assert np.all((u >= 0.0) & (u < 1.0))
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))     # exact multiples of 2^-53
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / len(u))
    counts, _ = np.histogram(u, bins=10, range=(0, 1))
    assert counts.min() > 300 and counts.max() < 500


def _tile(seed, singular=False):
    A = np.random.default_rng(seed).standard_normal((8, 8))
    if singular:
        A[:, 3] = 0.0
    LU = A.copy()
    piv, zr = O.getrf(LU)
    return LU, piv, zr


@pytest.mark.parametrize("alpha", [10.0, 50.0, 90.0])
def test_lu_frequency_matches_alpha(alpha):
    LU, piv, zr = _tile(1)
    n = 3000
    lu = sum(O.decide(O.CRIT_RANDOM, alpha, LU, piv, zr, [1.0], None, None, seed=7, k=k).dec
             == O.DEC_LU for k in range(n))
    p = alpha / 100.0
    assert abs(lu / n - p) < 4 * np.sqrt(p * (1 - p) / n)


def test_limits_and_zero_pivot():
    LU, piv, zr = _tile(2)
    for k in range(50):
        assert O.decide(O.CRIT_RANDOM, 0.0, LU, piv, zr, [1.0], None, None, seed=3, k=k).dec == O.DEC_QR
        assert O.decide(O.CRIT_RANDOM, 100.0, LU, piv, zr, [1.0], None, None, seed=3, k=k).dec == O.DEC_LU
    LU, piv, zr = _tile(3, singular=True)
    assert zr >= 0
    assert O.decide(O.CRIT_RANDOM, 100.0, LU, piv, zr, [1.0], None, None, seed=3, k=0).dec == O.DEC_QR


def test_decision_and_margin_from_the_draw():
    LU, piv, zr = _tile(4)
    for k in range(20):
        u = O.random_draw(99, k)
        sd = O.decide(O.CRIT_RANDOM, 50.0, LU, piv, zr, [1.0], None, None, seed=99, k=k)
        assert sd.dec == (O.DEC_LU if u < 0.5 else O.DEC_QR)
        assert sd.margin == pytest.approx(np.log2(0.5 / u))


def test_random_run_solves():
    rng = np.random.default_rng(5)
    N, nb = 256, 32
    A = rng.standard_normal((N, N))
    b = A @ np.ones(N)
    x, f = O.solve(A, b, nb, O.CRIT_RANDOM, 50.0, seed=11)
    expect = [O.DEC_LU if O.random_draw(11, k) < 0.5 else O.DEC_QR for k in range(N // nb)]
    assert f.dec.tolist() == expect
    assert O.backward_error(A, x, b) <= 1e-12
