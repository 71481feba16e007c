"""Batched persistent solves against the single-system path and the oracle.

Bars: decisions identical to luqr_factor with the flat TS tree at the same nb (FP64);
solutions within 1e-9 relative of the single-system path; eta <= 1e-13 for FP64 and for
FP32 + refinement; a few systems checked against the oracle's decisions."""
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


def systems(sizes, seed0=0, scaled=()):
    out = []
    for i, N in enumerate(sizes):
        A = inputs.gaussian(N, seed0 + i).contiguous().t().contiguous().t()
        A = A.clone()
        if i in scaled:
            nb = 32
            A[:nb, :nb] *= 1e-6
        dA = A.cuda()
        b = (dA @ torch.ones(N, 1, dtype=torch.float64, device="cuda")).reshape(-1).contiguous()
        out.append((dA, b))
    return out


@pytest.mark.parametrize("crit,alpha", [("max", 100.0), ("max", 3000.0), ("mumps", 2.1)])
def test_batched_fp64_matches_single_path(crit, alpha):
    from paper_1401_5522_gb300 import batched, luqr
    sizes = [64, 100, 257, 300, 511, 640, 95, 200]
    nbs = [32, 64, 32, 64, 64, 32, 32, 64]
    sy = systems(sizes, scaled=(1, 4))
    bs = [b.clone() for _, b in sy]
    bt = batched.Batch([A for A, _ in sy], bs, nbs, crit, alpha, "fp64")
    bt.run()
    dec, status, iters, eta = bt.results()
    assert np.all(status == 0)
    for i, ((A, b), N, nb) in enumerate(zip(sy, sizes, nbs)):
        x1 = b.clone()
        h = luqr.factor(A, nb, crit, alpha, b=x1, tree="flat_ts")
        d1, _ = h.decisions()
        n = len(d1)
        assert np.array_equal(dec[i, :n], d1), (i, dec[i, :n], d1)
        assert np.all(dec[i, n:] == 255)
        xb = bs[i]
        assert (xb - x1).abs().max().item() <= 1e-9 * x1.abs().max().item()
        assert eta[i] <= 1e-13, (i, eta[i])
        Ah = A.cpu().numpy()
        assert O.backward_error(Ah, xb.cpu().numpy(), b.cpu().numpy()) <= 1e-13


def test_batched_decisions_match_oracle():
    from paper_1401_5522_gb300 import batched
    sizes = [200, 333]
    sy = systems(sizes, seed0=50, scaled=(0,))
    bs = [b.clone() for _, b in sy]
    bt = batched.Batch([A for A, _ in sy], bs, [32, 32], "max", 2000.0, "fp64")
    bt.run()
    dec, status, _, _ = bt.results()
    for i, (A, b) in enumerate(sy):
        f = O.factor(A.cpu().numpy(), None, 32, O.CRIT_MAX, 2000.0, tree=O.TREE_FLAT_TS)
        assert np.array_equal(dec[i, :f.n], f.dec)


def test_batched_fp32_refinement_reaches_fp64_accuracy():
    from paper_1401_5522_gb300 import batched
    rng = np.random.default_rng(3)
    sizes = [int(v) for v in rng.integers(64, 700, size=24)]
    nbs = [32 if N < 256 else 64 for N in sizes]
    sy = systems(sizes, seed0=100, scaled=(2, 7))
    bs = [b.clone() for _, b in sy]
    bt = batched.Batch([A for A, _ in sy], bs, nbs, "max", 100.0, "fp32", tol=1e-13, max_iter=10)
    bt.run()
    dec, status, iters, eta = bt.results()
    assert np.all(status == 0)
    assert np.all(eta <= 1e-13), eta
    assert np.all(iters >= 2)
    for i, (A, b) in enumerate(sy[:4]):
        assert O.backward_error(A.cpu().numpy(), bs[i].cpu().numpy(), b.cpu().numpy()) <= 1e-13


def test_autotuner_returns_a_candidate_per_bucket():
    from paper_1401_5522_gb300 import batched

    def make(N, seed):
        return systems([N], seed0=seed)[0]

    sizes = [80, 90, 300, 320]
    table = batched.autotune(sizes, make, samples=2, reps=1)
    assert set(table) == {batched.bucket_of(80), batched.bucket_of(300)}
    assert all(v in batched.CANDIDATES for v in table.values())


def test_batched_graph_replays_are_repeatable():
    """The batch keeps its own right-hand sides, so plain runs and CUDA-graph launches
    solve the same systems every time and agree bit for bit."""
    from paper_1401_5522_gb300 import batched
    sizes = [70, 130, 300, 64, 500]
    nbs = [32, 64, 32, 32, 64]
    sy = systems(sizes, seed0=40, scaled=(2,))
    for prec in ("fp64", "fp32"):
        bs = [b.clone() for _, b in sy]
        bt = batched.Batch([A for A, _ in sy], bs, nbs, "max", 100.0, prec)
        bt.run()
        ref = [b.clone() for b in bs]
        d0, s0, i0, e0 = bt.results()
        for _ in range(3):
            bt.run_graph()
            d1, s1, i1, e1 = bt.results()
            assert np.all(s1 == 0) and np.array_equal(d1, d0) and np.array_equal(i1, i0)
            for x, r in zip(bs, ref):
                assert torch.equal(x, r)
        assert np.all(e0 <= 1e-13)
        bt.close()
