"""Writes the oracle's decision sequences at the benchmarked sizes (tests/golden/large_*.json).

Calls only the oracle (oracle/luqr_oracle_mt, the threaded C++ restatement of Alg. 1-4 and
Eq. 2-4) and the seeded input recipes of paper_1401_5522_gb300/inputs.py; nothing here
touches the GPU library.  The GPU tests (tests/test_gpu_large_parity.py) regenerate each
input from the same recipe, check its fingerprint, run the GPU solver with the same options
and compare decisions and margins with the stored ones.

Usage:  python tests/golden/make_large.py [name ...]      (default: every missing file)
        python tests/golden/make_large.py --list
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CRIT = {"max": 0, "sum": 1, "mumps": 2, "force_lu": 3, "force_qr": 4, "random": 5}
TREE = {"flat_ts": 0, "binary_tt": 1, "grouped": 2}

# Benchmarked configurations: N = 16384, nb = 256 iid N(0,1) matrices with the Max, Sum
# and MUMPS criteria at one small and one paper-scale alpha, the literal 20 % diagonal-tile
# variant and one run-time injection; N = 32768, nb = 256 conditioned matrices (the solve
# the benchmark times) in float64 and float32.
C2 = dict(N=16384, nb=256)
C3 = dict(N=32768, nb=256, recipe="conditioned", kappa=1e5, seed=0, criterion="max",
          tree="binary_tt")
C3P = dict(C3, tree="grouped", group=4, tree_small="binary_tt", tree_switch=64)
RUNS = {
    "c2_max_a100_tt": dict(C2, recipe="gaussian", seed=0, criterion="max", alpha=100.0,
                           tree="binary_tt"),
    "c2_max_a6000_tt": dict(C2, recipe="gaussian", seed=0, criterion="max", alpha=6000.0,
                            tree="binary_tt"),
    "c2_sum_a1000_ts": dict(C2, recipe="gaussian", seed=1, criterion="sum", alpha=1000.0,
                            tree="flat_ts"),
    "c2_sum_a1e6_tt": dict(C2, recipe="gaussian", seed=1, criterion="sum", alpha=1e6,
                           tree="binary_tt"),
    "c2_mumps_a10_tt": dict(C2, recipe="gaussian", seed=2, criterion="mumps", alpha=10.0,
                            tree="binary_tt"),
    "c2_mumps_a2.1_grouped": dict(C2, recipe="gaussian", seed=2, criterion="mumps", alpha=2.1,
                                  tree="grouped", group=4),
    "c2_max_a6000_scaled_tt": dict(C2, recipe="gaussian_scaled", seed=0, criterion="max",
                                   alpha=6000.0, tree="binary_tt"),
    "c2_max_a6000_inject_tt": dict(C2, recipe="gaussian", seed=0, criterion="max", alpha=6000.0,
                                   tree="binary_tt", inject=[5]),
    "c3_fp64_a100": dict(C3, alpha=100.0, dtype="float64"),
    "c3_fp32_a100": dict(C3, alpha=100.0, dtype="float32"),
    # the benchmark's tree policy: grouped tree (groups of 4) while a step has 64 or more
    # sub-diagonal tiles, binary TT below
    "c3p_fp64_a100": dict(C3P, alpha=100.0, dtype="float64"),
    "c3p_fp32_a100": dict(C3P, alpha=100.0, dtype="float32"),
}


def make_input(cfg):
    """The input matrix of a run (float64 numpy, column-major), from the seeded recipes."""
    from paper_1401_5522_gb300 import inputs
    N, nb, seed = cfg["N"], cfg["nb"], cfg["seed"]
    if cfg["recipe"] == "gaussian":
        A = inputs.gaussian(N, seed)
    elif cfg["recipe"] == "gaussian_scaled":
        A = inputs.gaussian(N, seed)
        A = inputs.scale_diag_tiles(A, nb, inputs.choose_panels(N // nb, 0.2, seed), 1e-8)
    elif cfg["recipe"] == "conditioned":
        A = inputs.conditioned(N, cfg["kappa"], seed)
    else:
        raise ValueError(cfg["recipe"])
    return A.numpy()


def fingerprint(A):
    """32 entries at fixed pseudo-random positions (exact, as hex) and the float64 sum of
    the first eight columns: enough to tell whether a host regenerated the same matrix."""
    N = A.shape[0]
    rng = np.random.default_rng(12345)
    pos = rng.integers(0, N, size=(32, 2))
    return {"pos": pos.tolist(), "val": [float(A[i, j]).hex() for i, j in pos],
            "sum8": float(np.sum(A[:, :8]))}


def run(name):
    from oracle import luqr_oracle_mt as M
    cfg = RUNS[name]
    A = make_input(cfg)
    fp32 = cfg.get("dtype") == "float32"
    b = None if fp32 else A @ np.ones(A.shape[0])
    t = time.time()
    res = M.factor(A, b, cfg["nb"], CRIT[cfg["criterion"]], cfg["alpha"],
                   tree=TREE[cfg["tree"]], group=cfg.get("group", 4),
                   tree_small=TREE[cfg.get("tree_small", "flat_ts")],
                   tree_switch=cfg.get("tree_switch", 0),
                   mumps_mode=cfg.get("mumps_mode", 0), inject=cfg.get("inject", ()),
                   dtype=np.float32 if fp32 else np.float64)
    dt = time.time() - t
    eta = None
    if b is not None:   # the oracle's own solution of A x = A 1 and its backward error
        from oracle import luqr_oracle as O
        eta = O.backward_error(A, M.back_substitution(res), b)
    out = {"name": name, "config": cfg, "fingerprint": fingerprint(A),
           "dec": "".join(str(int(d)) for d in res.dec),
           "margin": [float(v) for v in res.margin], "lhs": [float(v) for v in res.lhs],
           "rhs": [float(v) for v in res.rhs], "eta": eta,
           "oracle": "oracle/luqr_oracle_mt.cpp", "threads": res.threads,
           "seconds": round(dt, 1), "host": platform.machine(),
           "writer": "tests/golden/make_large.py"}
    path = os.path.join(HERE, f"large_{name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(f"{name}: {out['dec']} ({dt:.0f} s, {res.threads} threads)", flush=True)


def main(argv):
    if "--list" in argv:
        for k, v in RUNS.items():
            print(k, v)
        return
    names = [a for a in argv if not a.startswith("-")] or \
        [k for k in RUNS if not os.path.exists(os.path.join(HERE, f"large_{k}.json"))]
    for name in names:
        run(name)


if __name__ == "__main__":
    main(sys.argv[1:])
