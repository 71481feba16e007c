"""Python binding of libluqr.so (the C interface declared in include/luqr.h).

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current CUDA stream.  If the
library has not been built this module raises; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libluqr.so")

# constants mirrored from include/luqr.h
OK, ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_SINGULAR, ERR_NONFINITE, ERR_TIMEOUT, ERR_NOT_CONVERGED = \
    0, -1, -2, -3, -4, -5, -6, -7
DEC_QR, DEC_LU, DEC_ABORTED = 0, 1, 2
MAX, SUM, MUMPS, FORCE_LU, FORCE_QR = 0, 1, 2, 3, 4
TREE_FLAT_TS, TREE_BINARY_TT, TREE_GROUPED = 0, 1, 2
PREC_FP64, PREC_FP32 = 0, 1

RANDOM = 5
CRITERIA = {"max": MAX, "sum": SUM, "mumps": MUMPS, "force_lu": FORCE_LU, "force_qr": FORCE_QR,
            "random": RANDOM}
TREES = {"flat_ts": TREE_FLAT_TS, "binary_tt": TREE_BINARY_TT, "grouped": TREE_GROUPED}
PRECISIONS = {"fp64": PREC_FP64, "fp32": PREC_FP32}
SPECULATE = {"off": 0, "mlp": 1, "repeat": 2}
MLP_FEATURES, MLP_PARAMS = 16, 5313


class LuqrError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})" if what else
                         f"{status_string(status)} ({status})")


class Options(ctypes.Structure):
    _fields_ = [("tree", ctypes.c_int), ("group", ctypes.c_int), ("precision", ctypes.c_int),
                ("mumps_mode", ctypes.c_int), ("forced", ctypes.POINTER(ctypes.c_uint8)),
                ("inject", ctypes.POINTER(ctypes.c_int)), ("n_inject", ctypes.c_int),
                ("fp32_kernels", ctypes.c_int), ("speculate", ctypes.c_int),
                ("log_features", ctypes.c_int), ("mlp_params", ctypes.c_void_p),
                ("norm_mode", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("lu_variant", ctypes.c_int), ("timeout_ms", ctypes.c_int),
                ("domain", ctypes.c_int), ("tree_small", ctypes.c_int),
                ("tree_switch", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


_lib = None

# name -> (restype, argtypes); every symbol of include/luqr.h
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIGS = {
    "luqr_factor": (ctypes.c_int, [_P, _I64, _P, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   ctypes.POINTER(Options), _P, ctypes.POINTER(_P)]),
    "luqr_solve": (ctypes.c_int, [_P, _P, ctypes.c_int, _I64, _P]),
    "luqr_refine": (ctypes.c_int, [_P, _P, _I64, _P, _P, ctypes.c_double, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), _P]),
    "luqr_refine_gmres": (ctypes.c_int, [_P, _P, _I64, _P, _P, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_double), _P]),
    "luqr_decisions": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_int)]),
    "luqr_accuracy": (ctypes.c_int, [_P, _P, _P, _P]),
    "luqr_debug_replay_skip": (ctypes.c_int, [_P, ctypes.c_int]),
    "luqr_debug_tc_skip": (ctypes.c_int, [ctypes.c_int]),
    "luqr_step_stats": (ctypes.c_int, [_P, _P, _P]),
    "luqr_factor_data": (ctypes.c_int, [_P, _P, _I64]),
    "luqr_sync": (ctypes.c_int, [_P]),
    "luqr_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int)]),
    "luqr_dims": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_I64),
                                 ctypes.POINTER(ctypes.c_int)]),
    "luqr_destroy": (None, [_P]),
    "luqr_profile": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "luqr_profile_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "luqr_profile_select": (ctypes.c_int, [ctypes.POINTER(ctypes.c_char_p), ctypes.c_int]),
    "luqr_profile_trace": (ctypes.c_int, [ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_float),
                                          ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_uint64),
                                          _I64]),
    "luqr_gemm_sub_f32": (ctypes.c_int, [_P, _I64, _P, _I64, _P, _I64, _I64, _I64, _I64, _P, _P]),
    "luqr_panel_test_noalloc": (ctypes.c_int, [_P, _I64, _I64, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_double, ctypes.c_int, _P, _P, _P]),
    "luqr_batched_create": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.POINTER(Options), ctypes.c_double, ctypes.c_int,
                                           ctypes.POINTER(_P)]),
    "luqr_batched_run": (ctypes.c_int, [_P, _P]),
    "luqr_batched_run_graph": (ctypes.c_int, [_P, _P]),
    "luqr_batched_results": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_int)]),
    "luqr_batched_destroy": (None, [_P]),
    "luqr_mlp_forward": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "luqr_mlp_grad": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P, _P]),
    "luqr_mlp_adam": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, ctypes.c_float, _P]),
    "luqr_features": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_int)]),
    "luqr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "luqr_version": (ctypes.c_char_p, []),
}


def lib():
    """Load libluqr.so (built in-tree by paper_1401_5522_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1401_5522_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_string(status):
    return lib().luqr_status_string(int(status)).decode()


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check_matrix(A):
    import torch
    if not (isinstance(A, torch.Tensor) and A.is_cuda and A.dtype == torch.float64 and A.dim() == 2):
        raise TypeError("A must be a 2-D float64 CUDA tensor")
    if A.shape[0] != A.shape[1]:
        raise ValueError("A must be square")
    if A.stride(0) != 1:
        raise ValueError("A must be column-major (stride(0) == 1); use inputs.* or A.t().contiguous().t()")
    return A.stride(1) if A.shape[1] > 1 else A.shape[0]


class Handle:
    """A factorization living on the GPU (owns the library handle)."""

    def __init__(self, ptr, N, nb, stream):
        self._h = ctypes.c_void_p(ptr)
        self.N = N
        self.nb = nb
        self._stream = stream
        n = ctypes.c_int()
        npad = ctypes.c_int64()
        prec = ctypes.c_int()
        lib().luqr_dims(self._h, ctypes.byref(n), ctypes.byref(npad), ctypes.byref(prec))
        self.n, self.npad, self.precision = n.value, npad.value, prec.value

    def _ptr(self):
        if not self._h:
            raise RuntimeError("handle already destroyed")
        return self._h

    def decisions(self):
        """(dec uint8[n], margin float64[n]); synchronises."""
        dec = np.zeros(self.n, dtype=np.uint8)
        mg = np.zeros(self.n, dtype=np.float64)
        nout = ctypes.c_int()
        st = lib().luqr_decisions(self._ptr(), dec.ctypes.data_as(_P), mg.ctypes.data_as(_P),
                                  ctypes.byref(nout))
        if st not in (OK,):
            raise LuqrError(st, "luqr_decisions")
        return dec, mg

    def features(self):
        """(features float32[n, 16], predicted uint8[n]) logged during the factorization."""
        feat = np.zeros((self.n, MLP_FEATURES), dtype=np.float32)
        pred = np.zeros(self.n, dtype=np.uint8)
        nout = ctypes.c_int()
        st = lib().luqr_features(self._ptr(), feat.ctypes.data_as(_P), pred.ctypes.data_as(_P),
                                 ctypes.byref(nout))
        if st != OK:
            raise LuqrError(st, "luqr_features")
        return feat, pred

    def accuracy(self):
        """(eta, HPL3, norms[4]) of the last refinement's solution (Sec. V-A), computed by the
        library from its FP64 GPU norms {||A||, ||b - A x||, ||x||, ||b||}."""
        eta = ctypes.c_double()
        hpl3 = ctypes.c_double()
        norms = np.zeros(4)
        st = lib().luqr_accuracy(self._ptr(), ctypes.byref(eta), ctypes.byref(hpl3),
                                 norms.ctypes.data_as(_P))
        if st != OK:
            raise LuqrError(st, "luqr_accuracy")
        return eta.value, hpl3.value, norms

    def step_stats(self):
        lhs = np.zeros(self.n)
        rhs = np.zeros(self.n)
        st = lib().luqr_step_stats(self._ptr(), lhs.ctypes.data_as(_P), rhs.ctypes.data_as(_P))
        if st != OK:
            raise LuqrError(st, "luqr_step_stats")
        return lhs, rhs

    def factor_data(self):
        """The transformed padded workspace as a float64 numpy array (npad x npad)."""
        out = np.zeros((self.npad, self.npad), dtype=np.float64, order="F")
        st = lib().luqr_factor_data(self._ptr(), out.ctypes.data_as(_P), self.npad)
        if st != OK:
            raise LuqrError(st, "luqr_factor_data")
        return out

    def info(self):
        st = ctypes.c_int()
        step = ctypes.c_int()
        row = ctypes.c_int()
        r = lib().luqr_info(self._ptr(), ctypes.byref(st), ctypes.byref(step), ctypes.byref(row))
        if r != OK:
            raise LuqrError(r, "luqr_info")
        return st.value, step.value, row.value

    def sync(self):
        return lib().luqr_sync(self._ptr())

    def solve(self, B, stream=None):
        """Second-pass solve in place on B (N or N x nrhs float64 CUDA, column-major)."""
        import torch
        if not (B.is_cuda and B.dtype == torch.float64):
            raise TypeError("B must be a float64 CUDA tensor")
        if B.dim() == 1:
            if not B.is_contiguous():
                raise ValueError("B must be contiguous")
            nrhs, ldb = 1, B.shape[0]
        else:
            if B.stride(0) != 1:
                raise ValueError("B must be column-major")
            nrhs, ldb = B.shape[1], max(B.stride(1), B.shape[0])
        st = lib().luqr_solve(self._ptr(), ctypes.c_void_p(B.data_ptr()), nrhs, ldb,
                              _stream_ptr(stream))
        if st != OK:
            raise LuqrError(st, "luqr_solve")
        return B

    def refine(self, A, b, x, tol=1e-13, max_iter=30, stream=None):
        """Iterative refinement; returns (status, iterations, eta)."""
        lda = _check_matrix(A)
        it = ctypes.c_int()
        eta = ctypes.c_double()
        st = lib().luqr_refine(self._ptr(), ctypes.c_void_p(A.data_ptr()), lda,
                               ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                               float(tol), int(max_iter), ctypes.byref(it), ctypes.byref(eta),
                               _stream_ptr(stream))
        return st, it.value, eta.value

    def refine_gmres(self, A, b, x, tol=1e-13, max_iter=10, restart=30, stream=None):
        """GMRES-IR; returns (status, total GMRES iterations, eta)."""
        lda = _check_matrix(A)
        it = ctypes.c_int()
        eta = ctypes.c_double()
        st = lib().luqr_refine_gmres(self._ptr(), ctypes.c_void_p(A.data_ptr()), lda,
                                     ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                     float(tol), int(max_iter), int(restart), ctypes.byref(it),
                                     ctypes.byref(eta), _stream_ptr(stream))
        return st, it.value, eta.value

    def close(self):
        if self._h:
            lib().luqr_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


NORM_MODE = {"exact": 0, "estimate": 1}


def factor(A, nb, criterion="max", alpha=100.0, b=None, tree="flat_ts", group=4,
           precision="fp64", mumps_mode=0, forced=None, inject=None, stream=None,
           fp32_kernels="default", speculate="off", mlp_params=None, log_features=False,
           norm_mode="exact", seed=0, lu_variant="A1", timeout_ms=0, domain=1,
           tree_small="flat_ts", tree_switch=0):
    """luqr_factor on a column-major float64 CUDA matrix; b (if given) is overwritten by x.

    speculate: "off", "mlp" (mlp_params: float32 CUDA tensor of MLP_PARAMS values, kept
    alive by the caller until the factorization has run) or "repeat".
    norm_mode: "exact" ||A_kk^-1||_1 or "estimate" (Hager-Higham).
    criterion "random": LU with probability alpha/100 per step (SplitMix64 draws from seed).
    lu_variant: "A1" (GETRF of the diagonal tile) or "A2" (GEQRT of the diagonal tile).
    domain: tiles of the diagonal pivot domain (1: pivoting inside the diagonal tile).
    tree_small, tree_switch: steps with fewer than tree_switch sub-diagonal tiles use the
    tree tree_small (0: `tree` at every step)."""
    N = A.shape[0]
    lda = _check_matrix(A)
    crit = CRITERIA[criterion] if isinstance(criterion, str) else int(criterion)
    opt = Options()
    opt.tree = TREES[tree] if isinstance(tree, str) else int(tree)
    opt.group = int(group)
    opt.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    opt.mumps_mode = int(mumps_mode)
    opt.norm_mode = NORM_MODE[norm_mode] if isinstance(norm_mode, str) else int(norm_mode)
    opt.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    opt.timeout_ms = int(timeout_ms)
    opt.domain = int(domain)
    opt.tree_small = TREES[tree_small] if isinstance(tree_small, str) else int(tree_small)
    opt.tree_switch = int(tree_switch)
    opt.lu_variant = {"A1": 0, "A2": 1}[lu_variant] if isinstance(lu_variant, str) else int(lu_variant)
    opt.fp32_kernels = {"default": 0, "cuda": 1, "tensor": 2}[fp32_kernels]
    opt.speculate = SPECULATE[speculate] if isinstance(speculate, str) else int(speculate)
    opt.log_features = 1 if log_features else 0
    if mlp_params is not None:
        import torch
        if not (mlp_params.is_cuda and mlp_params.dtype == torch.float32 and
                mlp_params.is_contiguous() and mlp_params.numel() == MLP_PARAMS):
            raise TypeError(f"mlp_params must be a contiguous float32 CUDA tensor of {MLP_PARAMS}")
        opt.mlp_params = mlp_params.data_ptr()
    keep = []
    if forced is not None:
        fa = np.ascontiguousarray(np.asarray(forced, dtype=np.uint8))
        keep.append(fa)
        opt.forced = fa.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    if inject:
        ia = np.ascontiguousarray(np.asarray(list(inject), dtype=np.int32))
        keep.append(ia)
        opt.inject = ia.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        opt.n_inject = len(ia)
    bptr = None
    if b is not None:
        import torch
        if not (b.is_cuda and b.dtype == torch.float64 and b.is_contiguous() and b.numel() == N):
            raise TypeError("b must be a contiguous float64 CUDA vector of length N")
        bptr = ctypes.c_void_p(b.data_ptr())
    out = ctypes.c_void_p()
    st = lib().luqr_factor(ctypes.c_void_p(A.data_ptr()), lda, bptr, N, int(nb), crit,
                           float(alpha), ctypes.byref(opt), _stream_ptr(stream), ctypes.byref(out))
    if st != OK:
        raise LuqrError(st, "luqr_factor")
    return Handle(out.value, N, nb, stream)


def version():
    return lib().luqr_version().decode()


def profile(enable=True, reset=True, trace=False):
    """Start (or stop) the library's per-launch CUDA-event profiler; trace=True also keeps
    every launch's start and end (see profile_trace)."""
    mode = (2 if trace else 1) if enable else 0
    st = lib().luqr_profile(mode, 1 if reset else 0)
    if st != OK:
        raise LuqrError(st, "luqr_profile")
    return st


def profile_select(names=None):
    """Time only the launches of these kernel names (others are counted); None: all."""
    names = list(names or [])
    arr = (ctypes.c_char_p * max(len(names), 1))(*[n.encode() for n in names])
    st = lib().luqr_profile_select(arr, len(names))
    if st != OK:
        raise LuqrError(st, "luqr_profile_select")
    return st


def profile_trace():
    """Launch timeline of trace mode: list of (kernel name, start ms, end ms, stream id)."""
    L = lib()
    n = L.luqr_profile_trace(None, None, None, None, 0)
    names = (ctypes.c_char_p * max(n, 1))()
    t0 = (ctypes.c_float * max(n, 1))()
    t1 = (ctypes.c_float * max(n, 1))()
    sid = (ctypes.c_uint64 * max(n, 1))()
    n = min(n, L.luqr_profile_trace(names, t0, t1, sid, n))
    return [(names[i].decode(), float(t0[i]), float(t1[i]), int(sid[i])) for i in range(n)]


def profile_read(cap=64):
    """{kernel name: (launches, total_ms)} recorded since the last reset (synchronises)."""
    L = lib()
    names = (ctypes.c_char_p * cap)()
    launches = (ctypes.c_int64 * cap)()
    ms = (ctypes.c_double * cap)()
    n = L.luqr_profile_read(names, launches, ms, cap)
    return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(n)}


def gemm_sub_f32(C, A, B, status=None, stream=None):
    """C <- C - A B on the tensor cores (FP32, column-major CUDA tensors)."""
    import torch
    for t in (C, A, B):
        if not (t.is_cuda and t.dtype == torch.float32 and t.dim() == 2 and t.stride(0) == 1):
            raise TypeError("C, A, B must be column-major float32 CUDA matrices")
    M, N = C.shape
    K = A.shape[1]
    ld = lambda t: max(t.stride(1), t.shape[0])
    st = lib().luqr_gemm_sub_f32(ctypes.c_void_p(C.data_ptr()), ld(C), ctypes.c_void_p(A.data_ptr()),
                                 ld(A), ctypes.c_void_p(B.data_ptr()), ld(B), M, N, K,
                                 None if status is None else ctypes.c_void_p(status.data_ptr()),
                                 _stream_ptr(stream))
    if st != OK:
        raise LuqrError(st, "luqr_gemm_sub_f32")
    return C


def panel_test_noalloc(panel, nb, criterion="max", alpha=100.0, mumps_mode=0, dec=None,
                       margin=None, stream=None):
    """Allocation-free robustness test of one panel (rows x nb, column-major float64 CUDA).

    ``dec`` (uint8[1]) and ``margin`` (float64[1]) are caller-provided CUDA tensors on the
    panel's device that receive the result; the call itself allocates no device memory."""
    import torch
    if not (isinstance(panel, torch.Tensor) and panel.is_cuda and panel.dtype == torch.float64
            and panel.dim() == 2 and panel.stride(0) == 1):
        raise TypeError("panel must be a 2-D column-major float64 CUDA matrix")
    rows, cols = panel.shape
    if cols < nb:
        raise ValueError(f"panel has {cols} columns, fewer than nb = {nb}")
    if cols > 1 and panel.stride(1) < rows:
        raise ValueError("panel's column stride is smaller than its row count")
    ld = panel.stride(1) if cols > 1 else rows
    if dec is None or margin is None:
        raise TypeError("dec (uint8 CUDA[1]) and margin (float64 CUDA[1]) are required")
    if not (dec.is_cuda and dec.dtype == torch.uint8 and margin.is_cuda and
            margin.dtype == torch.float64):
        raise TypeError("dec must be a uint8 and margin a float64 CUDA tensor")
    if panel.device != dec.device or panel.device != margin.device:
        raise ValueError("panel, dec and margin must live on the same device")
    crit = CRITERIA[criterion] if isinstance(criterion, str) else int(criterion)
    with torch.cuda.device(panel.device):
        st = lib().luqr_panel_test_noalloc(ctypes.c_void_p(panel.data_ptr()), ld, rows, int(nb),
                                           crit, float(alpha), int(mumps_mode),
                                           ctypes.c_void_p(dec.data_ptr()),
                                           ctypes.c_void_p(margin.data_ptr()), _stream_ptr(stream))
    if st != OK:
        raise LuqrError(st, "luqr_panel_test_noalloc")
    return dec, margin


def _f32_cuda(t, what):
    import torch
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{what} must be a contiguous float32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def mlp_forward(params, X, out=None, stream=None):
    """Logits of the decision MLP for X (B x 16 float32 CUDA)."""
    import torch
    B = X.shape[0]
    if out is None:
        out = torch.empty(B, dtype=torch.float32, device=X.device)
    st = lib().luqr_mlp_forward(_f32_cuda(params, "params"), _f32_cuda(X, "X"),
                                _f32_cuda(out, "out"), B, _stream_ptr(stream))
    if st != OK:
        raise LuqrError(st, "luqr_mlp_forward")
    return out


def mlp_grad(params, X, y, grad, loss=None, stream=None):
    """Adds the mean-BCE gradient over (X, y) to grad (and the loss to loss[0])."""
    st = lib().luqr_mlp_grad(_f32_cuda(params, "params"), _f32_cuda(X, "X"), _f32_cuda(y, "y"),
                             X.shape[0], _f32_cuda(grad, "grad"),
                             None if loss is None else _f32_cuda(loss, "loss"), _stream_ptr(stream))
    if st != OK:
        raise LuqrError(st, "luqr_mlp_grad")
    return grad


def mlp_adam(params, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """One Adam step at iteration t >= 1 (in place on params, m, v)."""
    st = lib().luqr_mlp_adam(_f32_cuda(params, "params"), _f32_cuda(grad, "grad"), _f32_cuda(m, "m"),
                             _f32_cuda(v, "v"), int(t), float(lr), float(beta1), float(beta2),
                             float(eps), _stream_ptr(stream))
    if st != OK:
        raise LuqrError(st, "luqr_mlp_adam")
    return params
