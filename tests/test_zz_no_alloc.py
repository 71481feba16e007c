"""luqr_panel_test_noalloc: the per-step robustness test without device allocation.

Callers that cannot allocate (code held to a fixed memory budget or to a pool that the
host application owns, latency-critical paths that must not wait on the allocator) use
this entry point; its scratch is a fixed device array.  The test calls it through the C interface twice in a row on the same
panel and checks both results against the decision and margin that luqr_factor (the
existing entry point) computes for the first step of a matrix with that first panel,
within the FP64 margin bar of the parity tests.  Further cases compare it with the
oracle's criterion on a panel cut from a larger buffer (leading dimension > rows), at the
largest tile size, with the cumulative MUMPS reading, and check the aborted result of a
non-finite panel.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL_MARGIN = 1e-9


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1401_5522_gb300 import build
    build.build()


def colmajor(M):
    return torch.from_numpy(np.asfortranarray(M)).cuda()


@pytest.mark.parametrize("crit,alpha", [("max", 3000.0), ("sum", 1e5), ("mumps", 2.1),
                                        ("max", 1e9)])
def test_noalloc_panel_test_matches_factor(crit, alpha):
    from paper_1401_5522_gb300 import inputs, luqr
    N, nb = 1024, 128
    A = inputs.gaussian(N, seed=21).numpy()
    dA = colmajor(A)
    h = luqr.factor(dA, nb, crit, alpha)
    dec_ref, mg_ref = h.decisions()
    h.close()
    panel = dA[:, :nb]
    dec = torch.full((1,), 7, dtype=torch.uint8, device="cuda")
    mg = torch.full((1,), -12345.0, dtype=torch.float64, device="cuda")
    for _ in range(2):                                   # two calls in a row
        L = luqr.lib()
        st = L.luqr_panel_test_noalloc(ctypes.c_void_p(panel.data_ptr()), N, N, nb,
                                       luqr.CRITERIA[crit], alpha, 0,
                                       ctypes.c_void_p(dec.data_ptr()),
                                       ctypes.c_void_p(mg.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == luqr.OK
        torch.cuda.synchronize()
        assert int(dec.item()) == int(dec_ref[0])
        m = float(mg.item())
        if np.isfinite(mg_ref[0]):
            assert abs(m - mg_ref[0]) <= TOL_MARGIN
        else:
            assert m == mg_ref[0]
        dec.fill_(7)
        mg.fill_(-12345.0)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1401_5522_gb300 import luqr
    dummy = torch.zeros(2, dtype=torch.float64, device="cuda")
    L = luqr.lib()
    big_nb = L.luqr_panel_test_noalloc(ctypes.c_void_p(dummy.data_ptr()), 512, 512, 512, 0, 1.0, 0,
                                       ctypes.c_void_p(dummy.data_ptr()),
                                       ctypes.c_void_p(dummy.data_ptr()), None)
    too_tall = L.luqr_panel_test_noalloc(ctypes.c_void_p(dummy.data_ptr()), 32 * 2048, 32 * 2048, 32,
                                         0, 1.0, 0, ctypes.c_void_p(dummy.data_ptr()),
                                         ctypes.c_void_p(dummy.data_ptr()), None)
    assert big_nb == luqr.ERR_INVALID and too_tall == luqr.ERR_INVALID


def _call(panel, ld, rows, nb, crit, alpha, mode, dec, mg):
    from paper_1401_5522_gb300 import luqr
    return luqr.lib().luqr_panel_test_noalloc(
        ctypes.c_void_p(panel.data_ptr()), ld, rows, nb, luqr.CRITERIA[crit], alpha, mode,
        ctypes.c_void_p(dec.data_ptr()), ctypes.c_void_p(mg.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("nb,crit,alpha,mode", [(256, "max", 1e4, 0), (64, "mumps", 3e5, 1),
                                                (128, "sum", 2e5, 0)])
def test_noalloc_strided_subpanel_matches_oracle(nb, crit, alpha, mode):
    """A panel cut from a larger column-major buffer (ld > rows), against the oracle's
    step-0 criterion on the same values (tile norms, GETRF, exact inverse norm, Eq. 2-4)."""
    from oracle import luqr_oracle as O
    from paper_1401_5522_gb300 import inputs
    rows = 6 * nb
    big = inputs.gaussian(rows + 40, seed=33).numpy()
    P = big[17:17 + rows, 5:5 + nb].copy()
    norms = [O.norm1(P[i * nb:(i + 1) * nb]) for i in range(rows // nb)]
    local = np.max(np.abs(P[:nb]), axis=0)
    away = np.max(np.abs(P[nb:]), axis=0)
    LU = P[:nb].copy()
    piv, zr = O.getrf(LU)
    sd = O.decide({"max": O.CRIT_MAX, "sum": O.CRIT_SUM, "mumps": O.CRIT_MUMPS}[crit], alpha,
                  LU, piv, zr, norms[1:], local, away, mumps_mode=mode)
    dbig = colmajor(big)
    panel = dbig[17:17 + rows, 5:5 + nb]
    assert panel.stride(1) == rows + 40 > rows
    dec = torch.full((1,), 7, dtype=torch.uint8, device="cuda")
    mg = torch.zeros(1, dtype=torch.float64, device="cuda")
    from paper_1401_5522_gb300 import luqr
    for _ in range(2):
        assert _call(panel, panel.stride(1), rows, nb, crit, alpha, mode, dec, mg) == luqr.OK
        torch.cuda.synchronize()
        assert int(dec.item()) == sd.dec
        assert abs(float(mg.item()) - sd.margin) <= TOL_MARGIN
        dec.fill_(7)


def test_noalloc_nonfinite_panel_is_aborted():
    from paper_1401_5522_gb300 import inputs, luqr
    nb, rows = 64, 256
    P = inputs.gaussian(rows, seed=5).numpy()[:, :nb].copy()
    P[130, 7] = np.nan
    panel = colmajor(P)
    dec = torch.zeros(1, dtype=torch.uint8, device="cuda")
    mg = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _call(panel, rows, rows, nb, "max", 100.0, 0, dec, mg) == luqr.OK
    torch.cuda.synchronize()
    assert int(dec.item()) == luqr.DEC_ABORTED
    # the shared scratch keeps no state across calls: a clean panel afterwards decides normally
    P[130, 7] = 0.5
    panel.copy_(colmajor(P))
    assert _call(panel, rows, rows, nb, "max", 1e9, 0, dec, mg) == luqr.OK
    torch.cuda.synchronize()
    assert int(dec.item()) == luqr.DEC_LU


def test_noalloc_rejects_the_random_criterion():
    from paper_1401_5522_gb300 import luqr
    dummy = torch.zeros(64 * 64, dtype=torch.float64, device="cuda")
    dec = torch.zeros(1, dtype=torch.uint8, device="cuda")
    st = luqr.lib().luqr_panel_test_noalloc(ctypes.c_void_p(dummy.data_ptr()), 64, 64, 64,
                                            luqr.RANDOM, 50.0, 0, ctypes.c_void_p(dec.data_ptr()),
                                            ctypes.c_void_p(dummy.data_ptr()), None)
    assert st == luqr.ERR_INVALID
