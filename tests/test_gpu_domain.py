"""Diagonal-domain pivoting (Sec. II-B) on the GPU against the oracle's domain variant.

The Factor step pivots over tiles k .. k+d-1 (a tall GETRF); the criterion reads the
pivoted panel; an LU step applies the exchanges to columns k.. and b.  Bars as in the other
parity tests: identical decisions, margins to 1e-9 (FP64), triangle to 1e-10 x growth,
solution to 1e-9, eta <= 1e-13 (1e-12 for all-LU runs); the second pass on a new
right-hand side equals the oracle's replay.  With the whole panel as the domain and every
step LU the method is ordinary partial pivoting: U equals LAPACK dgetrf's.
"""
import numpy as np
import pytest
import scipy.linalg as sla
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


@pytest.mark.parametrize("d", [2, 4])
@pytest.mark.parametrize("tree", ["flat_ts", "binary_tt", "grouped"])
@pytest.mark.parametrize("crit,alpha", [("max", 2000.0), ("sum", 6000.0), ("mumps", 2.1)])
def test_domain_matches_oracle_fp64(d, tree, crit, alpha):
    from paper_1401_5522_gb300 import luqr
    N, nb = 520, 32
    A = inputs.gaussian(N, 3).numpy()
    b = A @ np.ones(N)
    x_o, f = O.solve(A, b, nb, CRIT[crit], alpha, tree=TREE[tree], group=3, domain=d)
    dA = colmajor(A)
    db = torch.from_numpy(b.copy()).cuda()
    h = luqr.factor(dA, nb, crit, alpha, b=db, tree=tree, group=3, domain=d)
    dec, mg = h.decisions()
    st, _, _ = h.info()
    assert st == 0
    assert np.array_equal(dec, f.dec), (dec, f.dec)
    fin = np.isfinite(f.margin)
    assert np.array_equal(np.isfinite(mg), fin)
    assert np.all(np.abs(mg[fin] - f.margin[fin]) <= 1e-9)
    x = db.cpu().numpy()
    assert O.backward_error(A, x, b) <= 1e-13
    assert np.max(np.abs(x - x_o.ravel())) <= 1e-9 * np.max(np.abs(x_o))
    W = h.factor_data()
    Ug = np.triu(W[:N, :N])
    rho = np.max(np.abs(f.U)) / np.max(np.abs(A))
    assert np.max(np.abs(Ug - f.U)) <= 1e-10 * max(1.0, rho) * np.max(np.abs(f.U))
    b2 = inputs.gaussian(N, 9).numpy()[:, 0].copy()
    y_o = O.replay_solve(f, b2).ravel()
    db2 = torch.from_numpy(b2.copy()).cuda()
    h.solve(db2)
    assert h.sync() == 0
    h.close()
    assert np.max(np.abs(db2.cpu().numpy() - y_o)) <= 1e-9 * np.max(np.abs(y_o))


def test_domain_admits_more_lu_steps_than_the_tile():
    from paper_1401_5522_gb300 import luqr
    N, nb = 512, 32
    A = inputs.gaussian(N, 4).numpy()
    dA = colmajor(A)
    lu = []
    for d in (1, 4):
        h = luqr.factor(dA, nb, "max", 2000.0, tree="binary_tt", domain=d)
        dec, _ = h.decisions()
        h.close()
        f = O.factor(A, None, nb, O.CRIT_MAX, 2000.0, tree=O.TREE_BINARY_TT, domain=d)
        assert np.array_equal(dec, f.dec)
        lu.append(int(dec.sum()))
    assert lu[1] >= lu[0]


def test_whole_panel_domain_all_lu_is_lapack_gepp():
    from paper_1401_5522_gb300 import luqr
    N, nb = 256, 32
    A = inputs.gaussian(N, 6).numpy()
    dA = colmajor(A)
    h = luqr.factor(dA, nb, "force_lu", 0.0, domain=N // nb)
    assert h.sync() == 0
    W = h.factor_data()
    h.close()
    lu, piv = sla.lu_factor(A)
    assert np.allclose(np.triu(W[:N, :N]), np.triu(lu), rtol=0, atol=1e-11 * np.abs(lu).max())


def test_domain_fp32_decisions_and_refinement():
    from paper_1401_5522_gb300 import luqr
    N, nb = 1024, 64
    A = inputs.gaussian(N, 5).numpy()
    b = A @ np.ones(N)
    f = O.factor(A, None, nb, O.CRIT_MAX, 2000.0, tree=O.TREE_BINARY_TT, dtype=np.float32,
                 domain=4)
    dA = colmajor(A)
    h = luqr.factor(dA, nb, "max", 2000.0, tree="binary_tt", precision="fp32", domain=4)
    dec, mg = h.decisions()
    fin = np.isfinite(f.margin)
    assert np.all(np.abs(f.margin[fin]) > 5e-2), "near-tie: comparison not meaningful"
    assert np.array_equal(dec, f.dec), (dec, f.dec)
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    st, its, eta = h.refine(dA, torch.from_numpy(b).cuda(), x, tol=1e-13, max_iter=30)
    h.close()
    assert st == 0 and eta <= 1e-13, (st, its, eta)


def test_domain_rejects_speculation_and_a2():
    from paper_1401_5522_gb300 import luqr
    dA = colmajor(np.eye(64))
    for kw in (dict(speculate="repeat"), dict(lu_variant="A2")):
        with pytest.raises(luqr.LuqrError) as e:
            luqr.factor(dA, 32, "max", 100.0, domain=2, **kw)
        assert e.value.status == luqr.ERR_INVALID
