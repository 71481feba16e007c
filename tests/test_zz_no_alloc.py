"""luqr_panel_test_noalloc: the per-step robustness test without device allocation.

Callers that cannot allocate (code recording a CUDA graph under stream capture, code held
to a fixed memory budget, latency-critical paths) use this entry point; its scratch is a
fixed device array.  The test calls it through the C interface twice in a row on the same
panel and checks both results against the decision and margin that luqr_factor (the
existing entry point) computes for the first step of a matrix with that first panel,
within the FP64 margin bar of the parity tests.  This file is collected last.
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
