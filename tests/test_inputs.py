"""The seeded input recipes behind the tests and the bench: layout, determinism and the
prescribed spectrum of the conditioned matrices."""
import numpy as np
import pytest
import torch

from paper_1401_5522_gb300 import inputs


@pytest.mark.parametrize("N", [64, 48])      # Walsh-Hadamard path, Haar path
@pytest.mark.parametrize("kappa", [1e2, 1e5, 1e8])
def test_conditioned_has_the_prescribed_singular_values(N, kappa):
    A = inputs.conditioned(N, kappa, seed=3)
    assert A.stride() == (1, N) and A.dtype == torch.float64
    sv = np.linalg.svd(A.numpy(), compute_uv=False)
    want = kappa ** (-np.arange(N) / (N - 1))
    assert np.allclose(sv, want, rtol=1e-9, atol=0.0)
    assert sv[0] / sv[-1] == pytest.approx(kappa, rel=1e-8)


def test_conditioned_is_dense_and_seeded():
    A = inputs.conditioned(64, 1e5, seed=1).numpy()
    B = inputs.conditioned(64, 1e5, seed=1).numpy()
    C = inputs.conditioned(64, 1e5, seed=2).numpy()
    assert np.array_equal(A, B) and not np.array_equal(A, C)
    assert np.count_nonzero(np.abs(A) < 1e-14) == 0          # no structural zeros


def test_gaussian_layout_and_moments():
    A = inputs.gaussian(256, 5)
    assert A.stride() == (1, 256)
    a = A.numpy().ravel()
    assert abs(a.mean()) < 4 / 256 and abs(a.std() - 1.0) < 0.02
    assert np.array_equal(inputs.gaussian(256, 5).numpy(), A.numpy())


def test_ones_rhs_is_row_sums():
    A = inputs.gaussian(32, 7)
    assert np.allclose(inputs.ones_rhs(A).numpy(), A.numpy().sum(axis=1), rtol=0, atol=1e-12)
