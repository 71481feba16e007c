"""Batched hybrid LU-QR solves (one persistent launch) and the tile-size autotuner.

Marshalling only: the solves run in libluqr.so's persistent kernel (luqr_batched_*).
The autotuner times that kernel itself, on sample systems drawn from each size bucket,
for every candidate tile size, and returns the faster tile size per bucket.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import luqr

BUCKETS = ((1, 128), (129, 256), (257, 384), (385, 512), (513, 768), (769, 1024), (1025, 8192))
CANDIDATES = (32, 64)


def _sigs():
    return luqr.lib()


class Batch:
    """A batch of systems (A_i column-major float64 CUDA tensors, b_i float64 CUDA vectors)."""

    def __init__(self, As, bs, nbs, criterion="max", alpha=100.0, precision="fp64", tol=1e-13,
                 max_iter=10, mumps_mode=0):
        L = _sigs()
        self.count = len(As)
        self._keep = (As, bs)
        for A in As:
            luqr._check_matrix(A)
            if A.stride(1) != A.shape[0]:
                raise ValueError("batched matrices must have lda == N")
        self.N = np.array([A.shape[0] for A in As], dtype=np.int32)
        self.nb = np.ascontiguousarray(np.asarray(nbs, dtype=np.int32))
        pa = (ctypes.c_void_p * self.count)(*[A.data_ptr() for A in As])
        pb = (ctypes.c_void_p * self.count)(*[b.data_ptr() for b in bs])
        opt = luqr.Options()
        opt.precision = luqr.PRECISIONS[precision]
        opt.mumps_mode = int(mumps_mode)
        crit = luqr.CRITERIA[criterion] if isinstance(criterion, str) else int(criterion)
        out = ctypes.c_void_p()
        st = L.luqr_batched_create(pa, pb, self.N.ctypes.data_as(ctypes.c_void_p),
                                   self.nb.ctypes.data_as(ctypes.c_void_p), self.count, crit,
                                   float(alpha), ctypes.byref(opt), float(tol), int(max_iter),
                                   ctypes.byref(out))
        if st != luqr.OK:
            raise luqr.LuqrError(st, "luqr_batched_create")
        self._h = out

    def run(self, stream=None):
        st = _sigs().luqr_batched_run(self._h, luqr._stream_ptr(stream))
        if st != luqr.OK:
            raise luqr.LuqrError(st, "luqr_batched_run")

    def run_graph(self, stream=None):
        """The same solve as one CUDA-graph launch (captured on the first call)."""
        st = _sigs().luqr_batched_run_graph(self._h, luqr._stream_ptr(stream))
        if st != luqr.OK:
            raise luqr.LuqrError(st, "luqr_batched_run_graph")

    def results(self):
        L = _sigs()
        nmax = ctypes.c_int()
        L.luqr_batched_results(self._h, None, None, None, None, ctypes.byref(nmax))
        dec = np.zeros((self.count, nmax.value), dtype=np.uint8)
        status = np.zeros(self.count, dtype=np.int32)
        iters = np.zeros(self.count, dtype=np.int32)
        eta = np.zeros(self.count, dtype=np.float64)
        st = L.luqr_batched_results(self._h, dec.ctypes.data_as(ctypes.c_void_p),
                                    status.ctypes.data_as(ctypes.c_void_p),
                                    iters.ctypes.data_as(ctypes.c_void_p),
                                    eta.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nmax))
        if st != luqr.OK:
            raise luqr.LuqrError(st, "luqr_batched_results")
        return dec, status, iters, eta

    def close(self):
        if self._h:
            _sigs().luqr_batched_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bucket_of(N):
    for i, (lo, hi) in enumerate(BUCKETS):
        if lo <= N <= hi:
            return i
    return len(BUCKETS) - 1


def autotune(sizes, make_system, criterion="max", alpha=100.0, precision="fp64", samples=24,
             reps=2, seed=0):
    """Tile size per size bucket, chosen by timing the persistent kernel.

    For each bucket that occurs in ``sizes``, ``samples`` systems of that bucket's sizes are
    built with ``make_system(N, seed) -> (A, b)`` and solved with every candidate nb; the
    candidate with the smallest median CUDA-event time wins.  Returns {bucket: nb}."""
    import torch
    rng = np.random.default_rng(seed)
    table = {}
    present = sorted({bucket_of(int(N)) for N in sizes})
    for bk in present:
        cand_sizes = [int(N) for N in sizes if bucket_of(int(N)) == bk]
        pick = [int(v) for v in rng.choice(cand_sizes, size=min(samples, len(cand_sizes)), replace=False)]
        systems = [make_system(N, 1000 + i) for i, N in enumerate(pick)]
        best = None
        for nb in CANDIDATES:
            times = []
            for _ in range(reps):
                bs = [b.clone() for _, b in systems]
                batch = Batch([A for A, _ in systems], bs, [nb] * len(pick), criterion, alpha,
                              precision)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                batch.run()
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
                batch.close()
            t = float(np.median(times))
            if best is None or t < best[1]:
                best = (nb, t)
        table[bk] = best[0]
    return table


def nb_for(sizes, table, default=64):
    return [table.get(bucket_of(int(N)), default) for N in sizes]
