"""The C-interface library builds, loads and exports every symbol include/luqr.h declares.

Runs without a GPU: only argument validation (which returns before any CUDA call)
and static strings are exercised.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1401_5522_gb300 import build, luqr
    build.build()
    return luqr.lib()


def declared_symbols():
    syms = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if not name.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", name)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        syms |= set(re.findall(r"\b(luqr_[a-z0-9_]+)\s*\(", text))
    return syms


def test_every_declared_symbol_is_exported(L):
    syms = declared_symbols()
    assert "luqr_factor" in syms and "luqr_solve" in syms and "luqr_decisions" in syms
    for s in sorted(syms):
        assert hasattr(L, s), s


def test_binding_declares_every_symbol():
    from paper_1401_5522_gb300 import luqr
    assert declared_symbols() <= set(luqr._SIGS)


def test_library_targets_sm_103a(L):
    from paper_1401_5522_gb300 import luqr
    assert "sm_103a" in luqr.version()


def test_status_strings(L):
    from paper_1401_5522_gb300 import luqr
    assert luqr.status_string(luqr.ERR_SINGULAR).startswith("singular")
    assert luqr.status_string(123) == "unknown status"


@pytest.mark.parametrize("N,nb,lda,alpha,crit", [
    (0, 64, 1, 1.0, 0),          # N < 1
    (100, 48, 100, 1.0, 0),      # nb not a multiple of 32
    (100, 1024, 100, 1.0, 0),    # nb too large
    (100, 64, 50, 1.0, 0),       # lda < N
    (100, 64, 100, -1.0, 0),     # alpha < 0
    (100, 64, 100, float("nan"), 0),
    (100, 64, 100, 1.0, 9),      # unknown criterion
])
def test_invalid_arguments_rejected_before_any_device_work(L, N, nb, lda, alpha, crit):
    from paper_1401_5522_gb300 import luqr
    out = ctypes.c_void_p(123)
    fake_dA = ctypes.c_void_p(0x1000)   # never dereferenced: validation fails first
    st = L.luqr_factor(fake_dA, lda, None, N, nb, crit, alpha, None, None, ctypes.byref(out))
    assert st == luqr.ERR_INVALID
    assert not out.value


def test_null_matrix_and_null_handle(L):
    from paper_1401_5522_gb300 import luqr
    out = ctypes.c_void_p()
    assert L.luqr_factor(None, 10, None, 10, 32, 0, 1.0, None, None, ctypes.byref(out)) == luqr.ERR_INVALID
    assert L.luqr_sync(None) == luqr.ERR_INVALID
    assert L.luqr_solve(None, None, 1, 1, None) == luqr.ERR_INVALID
    L.luqr_destroy(None)


def test_bad_options_rejected(L):
    from paper_1401_5522_gb300 import luqr
    opt = luqr.Options()
    opt.tree = 7
    out = ctypes.c_void_p()
    assert L.luqr_factor(ctypes.c_void_p(0x1000), 64, None, 64, 32, 0, 1.0, ctypes.byref(opt),
                         None, ctypes.byref(out)) == luqr.ERR_INVALID


@pytest.mark.parametrize("field,value", [("norm_mode", 2), ("norm_mode", -1), ("speculate", 3),
                                         ("speculate", 1), ("mumps_mode", 2), ("tree", 3),
                                         ("precision", 2), ("fp32_kernels", 3)])
def test_invalid_options_rejected_before_any_device_work(L, field, value):
    # speculate = 1 without mlp_params is invalid too
    from paper_1401_5522_gb300 import luqr
    opt = luqr.Options()
    setattr(opt, field, value)
    out = ctypes.c_void_p(123)
    st = L.luqr_factor(ctypes.c_void_p(0x1000), 100, None, 100, 64, 0, 1.0, ctypes.byref(opt),
                       None, ctypes.byref(out))
    assert st == luqr.ERR_INVALID
    assert not out.value


def test_unknown_criterion_after_random_rejected(L):
    from paper_1401_5522_gb300 import luqr
    out = ctypes.c_void_p(123)
    assert L.luqr_factor(ctypes.c_void_p(0x1000), 100, None, 100, 64, luqr.RANDOM + 1, 50.0,
                         None, None, ctypes.byref(out)) == luqr.ERR_INVALID


def test_options_layout_matches_header(L):
    # the binding's struct mirrors luqr_options: same size as the header's fields imply
    from paper_1401_5522_gb300 import luqr
    names = [f[0] for f in luqr.Options._fields_]
    assert names[-1] == "reserved" and "seed" in names and "norm_mode" in names
    text = open(os.path.join(ROOT, "include", "luqr.h")).read()
    body = text[text.index("typedef struct luqr_options {"):text.index("} luqr_options;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b([a-z_0-9]+)\s*(?:\[\d+\])?\s*;", body)
    assert fields == names


def test_profiler_argument_checks(L):
    from paper_1401_5522_gb300 import luqr
    assert L.luqr_profile(3, 0) == luqr.ERR_INVALID
    assert L.luqr_profile(-1, 0) == luqr.ERR_INVALID
    assert L.luqr_profile_select(None, 1) == luqr.ERR_INVALID
    assert L.luqr_profile_select(None, -1) == luqr.ERR_INVALID
    assert L.luqr_profile_select(None, 0) == luqr.OK
