"""Low-precision factorization + FP64 refinement on the conditioned matrices of the
mixed-precision workload (A = U diag(s) V^T, s geometric from 1 to 1/kappa).

Bar: the normwise backward error of the refined solution is <= 1e-13, computed by the
library (FP64 on the GPU) and recomputed on the host by the oracle's definition."""
import numpy as np
import pytest
import torch

from oracle import luqr_oracle as O
from paper_1401_5522_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1401_5522_gb300 import build
    build.build()


def setup(N, kappa, seed=0):
    A = inputs.conditioned(N, kappa, seed=seed, device="cuda")
    b = (A @ torch.ones(N, 1, dtype=torch.float64, device="cuda")).reshape(-1).contiguous()
    return A, b


@pytest.mark.parametrize("kappa", [1e2, 1e5])
@pytest.mark.parametrize("tree", ["binary_tt", "flat_ts"])
def test_fp32_factor_classic_refinement(kappa, tree):
    from paper_1401_5522_gb300 import luqr
    N, nb = 2048, 256
    A, b = setup(N, kappa)
    h = luqr.factor(A, nb, "max", 100.0, precision="fp32", tree=tree)
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    st, iters, eta = h.refine(A, b, x, tol=1e-13, max_iter=30)
    assert st == 0 and eta <= 1e-13, (st, iters, eta)
    An, bn, xn = A.cpu().numpy(), b.cpu().numpy(), x.cpu().numpy()
    assert O.backward_error(An, xn, bn) <= 1e-13


@pytest.mark.parametrize("kappa", [1e5, 1e6])
def test_fp32_factor_gmres_refinement(kappa):
    from paper_1401_5522_gb300 import luqr
    N, nb = 2048, 256
    A, b = setup(N, kappa, seed=1)
    h = luqr.factor(A, nb, "max", 100.0, precision="fp32", tree="binary_tt")
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    st, iters, eta = h.refine_gmres(A, b, x, tol=1e-13, max_iter=10, restart=60)
    assert st == 0 and eta <= 1e-13, (st, iters, eta)
    An, bn, xn = A.cpu().numpy(), b.cpu().numpy(), x.cpu().numpy()
    assert O.backward_error(An, xn, bn) <= 1e-13


def test_gmres_refinement_also_serves_fp64_factors():
    from paper_1401_5522_gb300 import luqr
    N, nb = 1024, 128
    A, b = setup(N, 1e6, seed=2)
    h = luqr.factor(A, nb, "max", 1e4, precision="fp64", tree="binary_tt")
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    st, iters, eta = h.refine_gmres(A, b, x, tol=1e-15, max_iter=5, restart=20)
    assert st == 0 and eta <= 1e-15 and iters <= 10, (st, iters, eta)


def test_kappa_1e8_through_fp64_factors():
    """kappa = 1e8 with a geometric spectrum leaves ~1/4 of the singular values below FP32
    resolution of A, so FP32 factors carry no information in those directions and
    restarted GMRES-IR stagnates; FP64 factors plus classic refinement reach the bar."""
    from paper_1401_5522_gb300 import luqr
    N, nb = 2048, 256
    A, b = setup(N, 1e8, seed=3)
    h = luqr.factor(A, nb, "max", 100.0, precision="fp64", tree="binary_tt")
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    st, iters, eta = h.refine(A, b, x, tol=1e-13, max_iter=5)
    assert st == 0 and eta <= 1e-13, (st, iters, eta)
    An, bn, xn = A.cpu().numpy(), b.cpu().numpy(), x.cpu().numpy()
    assert O.backward_error(An, xn, bn) <= 1e-13
