"""LU variant A2 (Sec. II-B) on the GPU against the oracle's A2 (lu_variant="A2").

The diagonal tile is factored by GEQRT: ||A_kk^-1||_1 = ||R^-1 Q^T||_1 (Eq. 2, 3), the
pivots of Eq. 4 are |R_jj|, and an LU step applies Q^T to A_kj and b_k, R^-1 to A_ik.
Bars as in the other parity tests: identical decisions, margins to 1e-9 (FP64), the
final triangle to 1e-10 x growth, the solution to 1e-9, eta <= 1e-13 (1e-12 for all-LU runs,
the tile-restricted "LU NoPiv" limit); the second pass on a new right-hand side equals the
oracle's replay; FP32 decisions against the float32 oracle (margins to the FP32 bar).
"""
import numpy as np
import pytest
import torch

from oracle import luqr_oracle as O
from paper_1401_5522_gb300 import inputs

pytestmark = pytest.mark.gpu

CRIT = {"max": O.CRIT_MAX, "sum": O.CRIT_SUM, "mumps": O.CRIT_MUMPS, "force_lu": O.CRIT_FORCE_LU}
TREE = {"flat_ts": O.TREE_FLAT_TS, "binary_tt": O.TREE_BINARY_TT, "grouped": O.TREE_GROUPED}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1401_5522_gb300 import build
    build.build()


def colmajor(M):
    return torch.from_numpy(np.asfortranarray(M)).cuda()


@pytest.mark.parametrize("tree", ["flat_ts", "binary_tt", "grouped"])
@pytest.mark.parametrize("crit,alpha", [("max", 2000.0), ("sum", 6000.0), ("mumps", 2.1),
                                        ("force_lu", 0.0)])
def test_a2_matches_oracle_fp64(tree, crit, alpha):
    from paper_1401_5522_gb300 import luqr
    N, nb = 512, 32
    A = inputs.gaussian(N, 3).numpy()
    b = A @ np.ones(N)
    x_o, f = O.solve(A, b, nb, CRIT[crit], alpha, tree=TREE[tree], group=3, lu_variant="A2")
    dA = colmajor(A)
    db = torch.from_numpy(b.copy()).cuda()
    h = luqr.factor(dA, nb, crit, alpha, b=db, tree=tree, group=3, lu_variant="A2")
    dec, mg = h.decisions()
    st, _, _ = h.info()
    assert st == 0
    assert np.array_equal(dec, f.dec), (dec, f.dec)
    if crit != "force_lu":
        assert 0 < int(dec.sum()) < len(dec)
    fin = np.isfinite(f.margin)
    assert np.array_equal(np.isfinite(mg), fin)
    assert np.all(np.abs(mg[fin] - f.margin[fin]) <= 1e-9)
    x = db.cpu().numpy()
    assert O.backward_error(A, x, b) <= (1e-12 if crit == "force_lu" else 1e-13)
    assert np.max(np.abs(x - x_o.ravel())) <= 1e-9 * np.max(np.abs(x_o))
    W = h.factor_data()
    Ug = np.triu(W[:N, :N])
    rho = np.max(np.abs(f.U)) / np.max(np.abs(A))
    assert np.max(np.abs(Ug - f.U)) <= 1e-10 * max(1.0, rho) * np.max(np.abs(f.U))
    # second pass on a new right-hand side (Sec. II-D): the stored A2 steps replayed
    b2 = inputs.gaussian(N, 9).numpy()[:, 0].copy()
    y_o = O.replay_solve(f, b2).ravel()
    db2 = torch.from_numpy(b2.copy()).cuda()
    h.solve(db2)
    torch.cuda.synchronize()
    assert np.max(np.abs(db2.cpu().numpy() - y_o)) <= 1e-9 * np.max(np.abs(y_o))
    h.close()


@pytest.mark.parametrize("kernels", ["tensor", "cuda"])
def test_a2_fp32_decisions_and_refinement(kernels):
    from paper_1401_5522_gb300 import luqr
    N, nb = 1024, 128
    A = inputs.gaussian(N, 5).numpy()
    b = A @ np.ones(N)
    f = O.factor(A, None, nb, O.CRIT_MAX, 3000.0, tree=O.TREE_BINARY_TT, dtype=np.float32,
                 lu_variant="A2")
    dA = colmajor(A)
    h = luqr.factor(dA, nb, "max", 3000.0, tree="binary_tt", precision="fp32",
                    fp32_kernels=kernels, lu_variant="A2")
    dec, mg = h.decisions()
    fin = np.isfinite(f.margin)
    assert np.all(np.abs(f.margin[fin]) > 5e-2), "near-tie: comparison not meaningful"
    assert np.array_equal(dec, f.dec), (dec, f.dec)
    assert np.all(np.abs(mg[fin] - f.margin[fin]) <= 5e-2)
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    st, its, eta = h.refine(dA, torch.from_numpy(b).cuda(), x, tol=1e-13, max_iter=30)
    h.close()
    assert st == 0 and eta <= 1e-13, (st, its, eta)
    assert O.backward_error(A, x.cpu().numpy(), b) <= 1e-13


def test_a2_rejects_estimate_and_speculation():
    from paper_1401_5522_gb300 import luqr
    dA = colmajor(np.eye(64))
    for kw in (dict(norm_mode="estimate"), dict(speculate="repeat")):
        with pytest.raises(luqr.LuqrError) as e:
            luqr.factor(dA, 32, "max", 100.0, lu_variant="A2", **kw)
        assert e.value.status == luqr.ERR_INVALID
