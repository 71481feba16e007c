"""The full-size configurations, in the launch configuration the bench times.

The oracle cannot factor these sizes, so each run is checked by properties that hold at
any size (normwise backward error after refinement, decisions of the speculative run equal
to those of the plain run) and by the one step the oracle can redo from the input alone:
step 0, whose panel is the input's first tile column (tile norms, GETRF of A_00 in the
factorization's precision, exact inverse norm, Eq. 2)."""
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


def L():
    from paper_1401_5522_gb300 import luqr
    return luqr


def step0_oracle(A, nb, alpha, dtype):
    """Step-0 decision of the Max criterion from the first tile column of A."""
    N = A.shape[0]
    n = N // nb
    P = A[:, :nb].cpu().numpy().astype(dtype)
    norms = [O.norm1(P[i * nb:(i + 1) * nb]) for i in range(n)]
    LU = P[:nb].copy()
    piv, zr = O.getrf(LU)
    return O.decide(O.CRIT_MAX, alpha, LU, piv, zr, norms[1:], None, None)


def refine_and_check(h, A, b, tol=1e-13):
    x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
    st, its, eta = h.refine(A, b, x, tol=tol, max_iter=30)
    assert st == 0, (st, its, eta)
    assert eta <= tol, eta
    return its


def test_headline_configuration_n32768():
    luqr = L()
    N, nb, alpha = 32768, 256, 100.0
    A = inputs.conditioned(N, 1e5, seed=0, device="cuda")
    b = (A @ torch.ones(N, 1, dtype=torch.float64, device="cuda")).reshape(-1).contiguous()
    h = luqr.factor(A, nb, "max", alpha, tree="binary_tt", precision="fp32")
    refine_and_check(h, A, b)
    dec, mg = h.decisions()
    lhs, rhs = h.step_stats()
    h.close()
    sd = step0_oracle(A, nb, alpha, np.float32)
    assert dec[0] == sd.dec
    assert abs(mg[0] - sd.margin) <= 1e-2            # FP32 GETRF, amplified by kappa(A_00)
    assert abs(rhs[0] - sd.rhs) <= 1e-12 * sd.rhs    # FP64 sums of the same FP32 values
    assert dec[-1] == L().DEC_LU                      # last step: nonsingular tile


def test_learned_speculation_configuration_n65536():
    """N = 65536, nb = 512, FP32 factorization + FP64 GMRES-IR, iid N(0,1) with 10% of
    the diagonal tiles scaled by 1e-8, Max alpha = 1e5, MLP speculation (the network
    trained by the library's kernels on logs of N = 4096 runs)."""
    from paper_1401_5522_gb300 import speculation as S
    luqr = L()
    N0, nb0 = 4096, 256
    runs = []
    for seed in range(6):
        A0 = inputs.gaussian(N0, 700 + seed, device="cuda")
        A0 = inputs.scale_diag_tiles(A0, nb0, inputs.choose_panels(N0 // nb0, 0.2, seed), 1e-8)
        runs.append(dict(A=A0, nb=nb0, criterion="max", alpha=(1e4, 1e5)[seed % 2],
                         precision="fp32", tree="binary_tt"))
    X, y = S.collect(runs)
    params, losses = S.train(X, y, epochs=150, batch=128, lr=3e-3)
    del runs
    N, nb, alpha = 65536, 512, 1e5
    n = N // nb
    A = inputs.gaussian(N, 5, device="cuda")
    A = inputs.scale_diag_tiles(A, nb, inputs.choose_panels(n, 0.1, 5), 1e-8)
    b = (A @ torch.ones(N, 1, dtype=torch.float64, device="cuda")).reshape(-1).contiguous()
    h = luqr.factor(A, nb, "max", alpha, tree="binary_tt", precision="fp32",
                    speculate="mlp", mlp_params=params)
    # LU steps admitted at alpha = 1e5 let the FP32 factors carry growth of that order, so
    # classic refinement stalls (kappa * growth * u_fp32 > 1): GMRES-IR, with the FP32
    # factorization as preconditioner, restores FP64 accuracy
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    st, its, eta = h.refine_gmres(A, b, x, tol=1e-13, max_iter=20, restart=40)
    assert st == 0 and eta <= 1e-13, (st, its, eta)
    dec, mg = h.decisions()
    _, pred = h.features()
    h.close()
    sd = step0_oracle(A, nb, alpha, np.float32)
    assert dec[0] == sd.dec
    if np.isfinite(sd.margin):
        assert abs(mg[0] - sd.margin) <= 1e-2
    print(f"\nN=65536 nb=512: LU fraction {np.mean(dec == 1):.3f}, "
          f"prediction accuracy {np.mean(pred == dec):.3f}, GMRES iterations {its}, eta {eta:.2e}")
