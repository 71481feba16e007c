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


@pytest.mark.parametrize("kappa,N", [(1e5, 2048), (1e2, 1000)])
def test_library_accuracy_equals_oracle_definition(kappa, N):
    """The library's eta and HPL3 (Sec. V-A), from its FP64 GPU norms, against the oracle's
    definitions evaluated on the host for the same x: they must agree to rounding of the
    norms (1e-2 relative is far below what a wrong norm, a dropped term or a 10x slip in
    the residual reduction would give)."""
    from paper_1401_5522_gb300 import luqr
    nb = 256
    if N & (N - 1):
        A = inputs.gaussian(N, 3).cuda()
        b = (A @ torch.ones(N, 1, dtype=torch.float64, device="cuda")).reshape(-1).contiguous()
    else:
        A, b = setup(N, kappa)
    h = luqr.factor(A, nb, "max", 100.0, precision="fp32", tree="binary_tt")
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    st, iters, eta = h.refine(A, b, x, tol=1e-13, max_iter=30)
    assert st == 0, (st, iters, eta)
    eta2, hpl3, norms = h.accuracy()
    h.close()
    An, bn, xn = A.cpu().numpy(), b.cpu().numpy(), x.cpu().numpy()
    eta_o = O.backward_error(An, xn, bn)
    hpl3_o = O.hpl3(An, xn, bn)
    assert eta2 == eta
    # the two residuals b - A x are each rounded at about u sum_j |a_ij x_j|, which is u in
    # eta's units: near eta ~ 5e-15 that alone is a few percent, hence the absolute 2u term
    u = 2.0 ** -53
    assert abs(eta - eta_o) <= 1e-2 * eta_o + 2 * u, (eta, eta_o)
    assert abs(hpl3 - hpl3_o) <= 1e-2 * hpl3_o + 2 * u / (u * An.shape[0]), (hpl3, hpl3_o)
    assert norms[0] == pytest.approx(np.max(np.sum(np.abs(An), axis=1)), rel=1e-13)
    assert norms[3] == pytest.approx(np.max(np.abs(bn)), rel=0)


def test_non_converged_refinement_returns_best_iterate():
    """max_iter = 0 from a coarse factorization: LUQR_ERR_NOT_CONVERGED, and the x handed
    back has the error reported (the best iterate), by the oracle's definition."""
    from paper_1401_5522_gb300 import luqr
    N, nb = 2048, 256
    A, b = setup(N, 1e5)
    h = luqr.factor(A, nb, "max", 100.0, precision="fp32", tree="binary_tt")
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    st, iters, eta = h.refine(A, b, x, tol=1e-300, max_iter=2)
    h.close()
    assert st == luqr.ERR_NOT_CONVERGED
    eta_o = O.backward_error(A.cpu().numpy(), x.cpu().numpy(), b.cpu().numpy())
    assert abs(eta - eta_o) <= 1e-2 * eta_o, (eta, eta_o)
