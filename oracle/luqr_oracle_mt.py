"""Threaded CPU oracle for the large configurations (binding of luqr_oracle_mt.cpp).

THIS MODULE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import it.  It never touches the GPU library.

``luqr_oracle_mt.cpp`` restates the same steps as ``luqr_oracle.py`` (Alg. 1-4, Eq. 2-4,
Sec. II-D) as plain C++ loops, threaded only over the independent columns of the
trailing matrix (and the rows of the TRSM), so that N = 16384 and N = 32768 runs finish
in minutes.  Its results do not depend on the thread count.  It covers the options of
the large configurations: Max / Sum / MUMPS (both readings) / forced / random criteria
with the exact inverse norm, the three trees, run-time injection, replayed decisions,
float64 or float32 storage and ragged N.  The diagonal-domain and A2 variants and the
inverse-norm estimate stay in ``luqr_oracle.py``.

Pins: ``tests/test_oracle_mt.py`` checks it against the pinned numpy oracle (decisions,
margins, transformed matrix) and directly against LAPACK GEPP (FORCE_LU, one tile),
numpy's Householder R (FORCE_QR, every tree), the worst-case matrix of Sec. III-A (all
LU with margin exactly 0) and thread-count invariance.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

from oracle.luqr_oracle import NonFinite, Singular

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "luqr_oracle_mt.cpp")
LIB = os.path.join(HERE, "libluqr_oracle_mt.so")
FLAGS = ["-O3", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-pthread"]

_lib = None


def build(force=False):
    """Compiles the C++ oracle in-tree with g++ (-O3 without contraction or fast-math: no
    floating-point reassociation)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp"
    r = subprocess.run(["g++", *FLAGS, "-o", tmp, SRC], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"g++ failed for {SRC}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        args = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                ctypes.c_int, ctypes.c_int,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_void_p, ctypes.c_void_p]
        for name in ("luqr_oracle_mt_factor_f64", "luqr_oracle_mt_factor_f32"):
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        for name in ("luqr_oracle_mt_backsolve_f64", "luqr_oracle_mt_backsolve_f32"):
            f = getattr(L, name)
            f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                          ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
            f.restype = ctypes.c_int
        L.luqr_oracle_mt_hardware_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def hardware_threads():
    return int(lib().luqr_oracle_mt_hardware_threads())


@dataclass
class Result:
    N: int
    nb: int
    n: int
    nrhs: int
    aug: np.ndarray          # N x (N + nrhs), Fortran order: the transformed [A | b]
    dec: np.ndarray          # uint8[n]; 255 past the last step run
    margin: np.ndarray
    lhs: np.ndarray
    rhs: np.ndarray
    steps: int               # steps run
    threads: int

    @property
    def U(self):
        return np.triu(self.aug[:, :self.N])


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def factor(A, b, nb, criterion, alpha, tree=0, group=4, mumps_mode=0, forced=None, inject=(),
           dtype=np.float64, seed=0, threads=None, steps=None, tree_small=0, tree_switch=0):
    """Alg. 1 on [A | b]; same arguments and decisions as luqr_oracle.factor.

    ``steps``: run only the first ``steps`` panels (a prefix); ``threads``: worker threads
    (default: every hardware thread).  Raises NonFinite / Singular like the numpy oracle.
    """
    A = np.asarray(A)
    N = A.shape[0]
    assert A.shape == (N, N)
    bb = np.zeros((N, 0)) if b is None else np.asarray(b).reshape(N, -1)
    nrhs = bb.shape[1]
    dtype = np.dtype(dtype)
    aug = np.empty((N, N + nrhs), dtype=dtype, order="F")
    aug[:, :N] = A
    aug[:, N:] = bb
    n = (N + nb - 1) // nb
    dec = np.zeros(n, dtype=np.uint8)
    margin = np.zeros(n)
    lhs = np.zeros(n)
    rhs = np.zeros(n)
    where = np.zeros(2, dtype=np.int32)
    done = np.zeros(1, dtype=np.int32)
    fz = None if forced is None else np.ascontiguousarray(np.asarray(forced, dtype=np.uint8))
    inj = np.ascontiguousarray(np.asarray(sorted(set(int(s) for s in inject)), dtype=np.int32))
    th = hardware_threads() if threads is None else int(threads)
    fn = lib().luqr_oracle_mt_factor_f64 if dtype == np.float64 else lib().luqr_oracle_mt_factor_f32
    assert dtype in (np.float64, np.float32)
    st = fn(_ptr(aug), N, N, N + nrhs, nb, int(criterion), float(alpha), int(tree), int(group),
            int(tree_small), int(tree_switch), int(mumps_mode), _ptr(fz), _ptr(inj) if len(inj) else None, len(inj), int(seed),
            th, -1 if steps is None else int(steps), _ptr(dec), _ptr(margin), _ptr(lhs), _ptr(rhs),
            _ptr(where), _ptr(done))
    if st == -5:
        raise NonFinite(int(where[0]))
    if st == -4:
        raise Singular(int(where[0]), int(where[1]))
    if st != 0:
        raise ValueError(f"oracle rejected the arguments (status {st})")
    return Result(N=N, nb=nb, n=n, nrhs=nrhs, aug=aug, dec=dec, margin=margin, lhs=lhs, rhs=rhs,
                  steps=int(done[0]), threads=th)


def back_substitution(res):
    """x = U^-1 c in float64 from a finished factorization (Sec. II-D)."""
    assert res.steps == res.n, "back substitution needs every step"
    x = np.zeros((res.N, res.nrhs), order="F")
    where = np.zeros(2, dtype=np.int32)
    fn = (lib().luqr_oracle_mt_backsolve_f64 if res.aug.dtype == np.float64
          else lib().luqr_oracle_mt_backsolve_f32)
    st = fn(_ptr(res.aug), res.N, res.N, res.nrhs, _ptr(x), res.N, _ptr(where))
    if st == -4:
        raise Singular(-1, int(where[1]))
    return x


def solve(A, b, nb, criterion, alpha, **kw):
    """Factor the augmented system and back-substitute; returns (x, Result)."""
    res = factor(A, b, nb, criterion, alpha, **kw)
    return back_substitution(res), res
