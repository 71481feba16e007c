#!/usr/bin/env python
"""Benchmark of the hybrid LU-QR solver on one or more GB300 GPUs.

Workload (default): N = 32768, nb = 256, A = U diag(s) V^T with s geometric from 1 to
1/kappa (kappa = 1e5) and U, V random orthogonal, b = A * ones; Max criterion,
alpha = 100, binary TT elimination tree.  One step = one solve to a normwise backward
error <= 1e-13: FP32 hybrid LU-QR factorization plus FP64 iterative refinement, all
in the library's CUDA kernels.  The metric is the solve time and the normalized
GFLOP/s (2N^3/3 per solve), next to the plain FP64 GPU solve of the same system.

One JSON line is printed by rank 0.  Under torchrun every rank solves its own
system (replicas, weak scaling); value aggregates all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "N=32768 solve time & GFLOP/s (2N^3/3) vs plain FP64 GPU at equal backward error"
FP32_FFMA_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FFMA lanes x 2 x max clock
FP64_DFMA_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12     # SMs x DFMA/clk x 2 x max clock


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="luqr", choices=["luqr", "reference"])
    p.add_argument("--N", type=int, default=32768)
    p.add_argument("--nb", type=int, default=256)
    p.add_argument("--kappa", type=float, default=1e5)
    p.add_argument("--criterion", default="max")
    p.add_argument("--alpha", type=float, default=100.0)
    # default tree policy: the fastest of the tuner's candidates on this GPU at N = 32768
    # (bench.py --tune-tree 1 re-times them)
    p.add_argument("--tree", default="grouped")
    p.add_argument("--tree-small", default="binary_tt",
                   help="tree of the steps with fewer than --tree-switch sub-diagonal tiles")
    p.add_argument("--tree-switch", type=int, default=64)
    p.add_argument("--group", type=int, default=4, help="group size of the grouped tree")
    p.add_argument("--tune-tree", type=int, default=0,
                   help="time candidate tree policies on the input (untimed setup) and use the "
                        "fastest")
    p.add_argument("--precision", default="fp32")
    p.add_argument("--tol", type=float, default=1e-13)
    p.add_argument("--fp32-kernels", default="default", choices=["default", "cuda", "tensor"])
    p.add_argument("--speculate", default="mlp", choices=["off", "repeat", "mlp"],
                   help="predicted-branch speculation of the factorization (mlp: the network "
                        "is trained at startup, outside the timed region)")
    p.add_argument("--fp64-baseline", type=int, default=3,
                   help="timed plain FP64 solves of the headline system (the speedup denominator)")
    p.add_argument("--e2e-steps", type=int, default=1)
    p.add_argument("--cpu-steps", type=int, default=1,
                   help="panels of the oracle's timed sample (per-step extrapolated)")
    p.add_argument("--forms", type=int, default=1,
                   help="also measure the batched and the MLP-speculative forms")
    p.add_argument("--batch-count", type=int, default=4096)
    p.add_argument("--configs", type=int, default=1,
                   help="also time the other configurations (C1, C2 subset, C3 kappa/alpha "
                        "variants, C5 speculation modes); one GPU only")
    p.add_argument("--seed", type=int, default=0)
    return p.parse_args(argv)


def tree_kw(args):
    """luqr.factor keywords of the tree policy."""
    return dict(tree=args.tree, tree_small=args.tree_small, tree_switch=args.tree_switch,
                group=args.group)


def tree_desc(args):
    def one(t):
        return f"{t} tree" + (f" (groups of {args.group})" if t == "grouped" else "")
    if args.tree_switch > 0:
        return (f"{one(args.tree)} from {args.tree_switch} sub-diagonal tiles, "
                f"{one(args.tree_small)} below")
    return one(args.tree)


# ------------------------------------------------------------------ flop model
def tree_at(tree, m):
    """The tree of a step with m sub-diagonal tiles: `tree` is a name, or a policy
    (tree, tree_small, tree_switch[, group]) that takes tree_small below tree_switch tiles."""
    if isinstance(tree, (tuple, list)):
        big, small, switch = tree[:3]
        return small if switch > 0 and m < switch else big
    return tree


def group_of(tree):
    return tree[3] if isinstance(tree, (tuple, list)) and len(tree) > 3 else 4


def tree_counts(tree, m):
    """(GEQRT singles, TS pairs, TT pairs) of a QR step with m sub-diagonal tiles, as the
    library's tile lists build them: flat TS 1 / m / 0; binary TT m+1 / 0 / m; grouped
    (groups of g tiles, H = ceil((m+1)/g) heads) H / m+1-H / H-1."""
    t = tree_at(tree, m)
    if t == "flat_ts":
        return 1, m, 0
    if t == "binary_tt":
        return m + 1, 0, m
    g = group_of(tree)
    H = (m + 1 + g - 1) // g
    return H, m + 1 - H, H - 1


def step_kernel_flops(dec, n, nb, tree, ncols_extra, replay=False):
    """Algorithmic flops per kernel class for one factorization (replay=False) or one
    second-pass solve on a single right-hand side (replay=True).  Per Table I:
    GEMM 2 nb^3 per tile pair, UNMQR 2 nb^3 per tile, TSMQR 4 nb^3, TTMQR 2 nb^3
    (triangular V), GEQRT 4/3 nb^3, TSQRT 2 nb^3, TTQRT 2/3 nb^3, TRSM nb^3."""
    out = {}

    def add(k, v):
        out[k] = out.get(k, 0.0) + v

    nb3 = float(nb) ** 3
    for k in range(n):
        m = n - 1 - k
        cols = 1.0 if replay else m * nb + ncols_extra
        if dec[k] == 1:
            if not replay:
                add("k_trsm", m * nb3)
            add("k_swptrsm", cols * nb * nb)
            add("k_gemm_update", 2.0 * m * nb * cols * nb)
        else:
            singles, ts, tt = tree_counts(tree, m)
            if not replay:
                add("k_geqrt", singles * 4.0 / 3.0 * nb3)
                add("k_tsqrt", ts * 2.0 * nb3)
                add("k_ttqrt", tt * 2.0 / 3.0 * nb3)
            add("k_unmqr", singles * 2.0 * nb * nb * cols)
            add("k_tsmqr", ts * 4.0 * nb * nb * cols)
            add("k_ttmqr", tt * 2.0 * nb * nb * cols)
        if not replay:
            add("k_getrf", 2.0 / 3.0 * nb3)
    return {k: v for k, v in out.items() if v}


def step_tc_bytes(dec, n, nb, tree, ncols_extra):
    """Algorithmic HBM bytes per tensor-core update kernel for one FP32 factorization:
    every launch reads its B operand and C (when accumulated), writes C, and reads its
    nb x nb FP32 A operand once.  W = V^T C (UNMQR) / W = C1 + V2^T C2 (TS/TT pair);
    C -= (V T^T) W; C1 -= T^T W; C2 -= (V2 T^T) W; LU: row k <- X row k (X = L^-1 P, in
    place) and C -= L U.  The tensor-core kernels update the bulk columns only: tile
    column k+1 goes through the look-ahead's CUDA-core kernels."""
    out = {}

    def add(k, v):
        out[k] = out.get(k, 0.0) + v

    a_op = 4.0 * nb * nb
    for k in range(n):
        m = n - 1 - k
        cols = (m - 1) * nb + ncols_extra
        if cols <= 0:
            continue
        if dec[k] == 1:
            rows = m * nb
            if cols >= 64 and nb <= 256:
                add("k_tc_lu_apply", 8.0 * nb * cols + a_op)
            add("k_tc_lu_gemm", 4.0 * (rows * nb + nb * cols + 2.0 * rows * cols))
            continue
        singles, ts, tt = tree_counts(tree, m)
        add("k_tc_unmqr_w", singles * (8.0 * nb * cols + a_op))
        add("k_tc_unmqr_c", singles * (12.0 * nb * cols + a_op))
        for kind, pairs in (("ts", ts), ("tt", tt)):
            if pairs:
                add(f"k_tc_{kind}mqr_w", pairs * (12.0 * nb * cols + a_op))
                add(f"k_tc_{kind}mqr_c1", pairs * (12.0 * nb * cols + a_op))
                add(f"k_tc_{kind}mqr_c2", pairs * (12.0 * nb * cols + a_op))
    return out


def update_work(dec, n, nb, tree, s_c):
    """Algorithmic work of the bulk trailing update (tile columns k+2.. and the right-hand
    side are the tensor-core kernel's; column k+1 is the look-ahead's) for one factorization:
    bytes = the trailing rows k.. x bulk columns read and written once per step (s_c bytes an
    element), flops = Table I's update flops on those columns (LU: SWPTRSM + GEMM; QR: UNMQR
    + TSMQR/TTMQR).  Returns (bytes, flops)."""
    by = fl = 0.0
    for k in range(n):
        m = n - 1 - k
        cols = (m - 1) * nb
        if cols <= 0:
            continue
        by += 2.0 * s_c * (m + 1) * nb * cols
        if dec[k] == 1:
            fl += nb * nb * cols + 2.0 * m * nb * nb * cols
        else:
            singles, ts, tt = tree_counts(tree, m)
            fl += (2.0 * singles + 4.0 * ts + 2.0 * tt) * nb * nb * cols
    return by, fl


# CUDA function behind each launch label of the library's profiler
KERNEL_OF_LABEL = {
    **{f"k_tc_{r}": "k_gemm_tc4" for r in ("ttmqr_w", "ttmqr_c1", "ttmqr_c2", "tsmqr_w",
                                            "tsmqr_c1", "tsmqr_c2", "unmqr_w", "unmqr_c",
                                            "lu_gemm", "lu_apply")},
    "k_tc_gram": "k_gemm_tc", "k_tc_vt": "k_gemm_tc",
    "k_ttqrt": "k_pair_qrt", "k_tsqrt": "k_pair_qrt",
    "k_ttmqr": "k_pair_apply", "k_tsmqr": "k_pair_apply",
}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per algorithmic byte (the
# trailing matrix read + written once per step) of the tensor-core update kernel, summed
# over the 535 launches of one N=8192 nb=256 FP32 solve (binary TT tree, 31 QR steps + 1 LU)
# captured with ncu: 30.06 GB against 5.44 GB.  ncu flushes the caches before each launch,
# so this is the cold-cache figure.  The ratio carries over to other sizes: each QR step
# makes the same passes (W, C and the pair passes of each tree level), and the levels of a
# binary tree touch (m+1)(1 + 1/2 + 1/4 ...) < 2(m+1) tile rows whatever the depth.
TRAFFIC_RATIO = {"k_gemm_tc4": 30.055 / 5.4447}


def traffic_per_launch(kernel, alg_bytes_per_launch):
    r = TRAFFIC_RATIO.get(kernel)
    return None if r is None else r * alg_bytes_per_launch


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "source": "fallback"}


TF32_PER_BF16 = 1.1 / 2.25      # nominal dense TF32 / BF16 tensor rates of the part


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle leg
def oracle_sample(A, args, steps=1):
    """Times the CPU oracle (the threaded C++ restatement, as it stands) on a bounded sample
    of the benchmarked solve: the first `steps` panels of the FP64 factorization of the same
    matrix on every host core, extrapolated to the whole solve by the Table I flops of the
    sampled steps against those of the full decision sequence (taken from the oracle's own
    decisions for the sampled steps and, beyond them, from the criterion's all-QR reading of
    alpha = 100 on these matrices: QR at every step but the last)."""
    import numpy as np
    from oracle import luqr_oracle as O
    from oracle import luqr_oracle_mt as M
    N, nb = A.shape[0], args.nb
    crit = {"max": O.CRIT_MAX, "sum": O.CRIT_SUM, "mumps": O.CRIT_MUMPS}[args.criterion]
    trees = {"flat_ts": 0, "binary_tt": 1, "grouped": 2}
    M.build()
    t0 = time.perf_counter()
    res = M.factor(A, None, nb, crit, args.alpha, tree=trees[args.tree], group=args.group,
                   tree_small=trees[args.tree_small], tree_switch=args.tree_switch, steps=steps)
    t = time.perf_counter() - t0
    n = res.n
    dec = np.zeros(n, dtype=np.uint8)
    dec[-1] = 1
    dec[:steps] = res.dec[:steps]
    f_all = sum(O.step_flops(int(d), n - 1 - k, nb) for k, d in enumerate(dec))
    f_smp = sum(O.step_flops(int(d), n - 1 - k, nb) for k, d in enumerate(dec[:steps]))
    t_full = t * f_all / f_smp
    return {"value": O.normalized_gflops(N, t_full), "seconds_sample": t, "steps": steps,
            "seconds_extrapolated": t_full, "N": N, "threads": res.threads,
            "nproc": os.cpu_count(), "sample_dec": [int(v) for v in res.dec[:steps]],
            "sample_margin": [float(v) for v in res.margin[:steps]]}


def cpu_baseline_dict(res, args):
    if "error" in res:
        return {"value": None, "unit": "GFLOP/s", "kind": "oracle", "error": res["error"]}
    return {"value": res.get("value"), "unit": "GFLOP/s", "cores": res.get("threads"),
            "nproc": res.get("nproc"), "kind": "oracle",
            "sample": (f"threaded C++ oracle (FP64, {res.get('threads')} threads on "
                       f"{res.get('nproc')} host cores), first {res.get('steps')} panel(s) of the "
                       f"N={res.get('N')}, nb={args.nb} solve of the same matrix in "
                       f"{res.get('seconds_sample', 0):.1f} s, per-step extrapolated by Table I "
                       f"flops to {res.get('seconds_extrapolated', 0):.0f} s per solve; "
                       f"GFLOP/s = (2/3)N^3/t"),
            "sample_decisions": res.get("sample_dec"), "sample_margins": res.get("sample_margin")}


def reference_arm(args, config):
    """The oracle timed as the reference arm: W warm-up samples on a small system, then K
    timed samples (first panels of the benchmarked solve, per-step extrapolated)."""
    import torch
    from paper_1401_5522_gb300 import inputs
    dev = "cuda" if torch.cuda.is_available() else "cpu"   # input recipe only; same bits
    small = inputs.conditioned(2048, args.kappa, seed=args.seed, device=dev).cpu().numpy()
    for _ in range(args.warmup):
        oracle_sample(small, args, steps=1)
    A = inputs.conditioned(args.N, args.kappa, seed=args.seed, device=dev).cpu().numpy()
    samples = [oracle_sample(A, args, steps=args.cpu_steps) for _ in range(max(args.steps, 1))]
    t_full = sum(r["seconds_extrapolated"] for r in samples) / len(samples)
    res = dict(samples[-1])
    res["value"] = (2.0 / 3.0) * float(args.N) ** 3 / t_full / 1e9
    res["seconds_extrapolated"] = t_full
    cfg = dict(config, N=args.N, oracle_sample=f"first {args.cpu_steps} panel(s) per step")
    return {"metric": METRIC, "impl": "reference", "value": res["value"], "unit": "GFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_full * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": cpu_baseline_dict(res, args),
            "e2e": {"value": res["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------ replicas
def job_rate(ms_local, world, flops_per_rank, device):
    """Whole-job rate of `world` replicas: every rank solves its own system; the job's time
    is the slowest rank's (max over ranks) and the value counts all ranks' work.
    Returns (ms_max, GFLOP/s)."""
    ms = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, flops_per_rank * world / (ms / 1e3) / 1e9


# ------------------------------------------------------------------ other forms
def batched_form(args, plain_ms_per_normflop=None):
    """4096 independent systems, N uniform in [64, 1024], iid N(0,1), 10% with a 1e-6-scaled
    leading tile; Max alpha=100; one persistent launch replayed as a CUDA graph; tile size
    per size bucket from the autotuner; FP64 and FP32 + FP64 refinement."""
    import numpy as np
    import torch
    from paper_1401_5522_gb300 import batched, inputs
    sizes = inputs.batch_sizes(args.batch_count, 64, 1024, args.seed + 4)
    scaled = set(inputs.choose_panels(args.batch_count, 0.1, args.seed + 4))
    As, bs = [], []
    for i, N in enumerate(sizes):
        A = inputs.gaussian(N, 10_000 + i, device="cuda")
        if i in scaled:
            A[:32, :32] *= 1e-6
        As.append(A)
        bs.append((A @ torch.ones(N, 1, dtype=torch.float64, device="cuda")).reshape(-1).contiguous())

    def make_system(N, seed):
        A = inputs.gaussian(N, seed, device="cuda").contiguous().t().contiguous().t()
        return A, (A @ torch.ones(N, 1, dtype=torch.float64, device="cuda")).reshape(-1).contiguous()

    table = batched.autotune(sizes, make_system, "max", 100.0, "fp64", samples=12, reps=1)
    nbs = batched.nb_for(sizes, table)
    flops = sum((2.0 / 3.0) * float(N) ** 3 for N in sizes)
    out = {"workload": f"{args.batch_count} systems, N~U[64,1024], iid N(0,1), 10% with a "
                       "1e-6-scaled leading tile, Max alpha=100, one persistent launch as a "
                       "CUDA graph", "nb_per_bucket": {str(k): v for k, v in table.items()}}
    for prec in ("fp64", "fp32"):
        xs = [b.clone() for b in bs]
        bt = batched.Batch(As, xs, nbs, "max", 100.0, prec, tol=1e-13, max_iter=10)
        bt.run_graph()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record()
        for _ in range(reps):
            bt.run_graph()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        dec, status, iters, eta = bt.results()
        bt.close()
        out[prec] = {"ms": ms, "gflops_normalized": flops / (ms / 1e3) / 1e9,
                     "max_eta": float(np.max(eta)), "failed": int(np.sum(status != 0)),
                     "mean_ir_iters": float(np.mean(iters)) if prec == "fp32" else 0.0,
                     "lu_fraction": float(np.mean(dec[dec != 255] == 1))}
    out["speedup_fp32_ir_over_fp64"] = out["fp64"]["ms"] / out["fp32"]["ms"]
    out["alu_peak_tflops"] = {"fp64": FP64_DFMA_PEAK_TFLOPS, "fp32": FP32_FFMA_PEAK_TFLOPS}
    del As, bs
    torch.cuda.empty_cache()
    return out


def train_decision_mlp(args):
    """Trains the decision MLP with the library's kernels on logged (features, decision)
    pairs from N=4096, nb=256 iid N(0,1) matrices with 20% of the diagonal tiles scaled
    by 1e-8 (Max alpha in {1e4, 3e4, 1e5}: paper-scale alpha, so both classes occur)."""
    import numpy as np
    from paper_1401_5522_gb300 import inputs
    from paper_1401_5522_gb300 import speculation as S
    N0, nb0 = 4096, 256
    runs = []
    for seed in range(48):   # 768 logged steps
        A0 = inputs.gaussian(N0, 500 + seed, device="cuda")
        A0 = inputs.scale_diag_tiles(A0, nb0, inputs.choose_panels(N0 // nb0, 0.2, seed), 1e-8)
        runs.append(dict(A=A0, nb=nb0, criterion="max", alpha=(1e4, 3e4, 1e5)[seed % 3],
                         precision="fp32", **tree_kw(args)))
    t0 = time.time()
    X, y = S.collect(runs)
    params, losses = S.train(X, y, epochs=200, batch=128, lr=3e-3)
    info = {"samples": int(len(y)), "lu_fraction": float(np.mean(y)),
            "loss_first": losses[0], "loss_last": losses[-1], "seconds": time.time() - t0}
    return params, info


def speculation_form(args, A, b, x, head_ms, params, train_info):
    """Times the headline solve with speculation off and with the repeat-previous predictor
    (decisions and results are the same in every mode)."""
    import numpy as np
    import torch
    from paper_1401_5522_gb300 import luqr
    out = {"training": train_info, "headline_mode": args.speculate}
    stream = torch.cuda.current_stream()
    modes = [("off", {}), ("repeat", {}), ("mlp", {"mlp_params": params})]
    for mode, extra in modes:
        if mode == args.speculate:
            continue
        def solve():
            h = luqr.factor(A, args.nb, args.criterion, args.alpha, **tree_kw(args),
                            precision=args.precision, fp32_kernels=args.fp32_kernels,
                            speculate=mode, **extra)
            st, its, eta = h.refine(A, b, x, tol=args.tol, max_iter=30)
            dec, _ = h.decisions()
            pred = h.features()[1] if mode != "off" else dec
            h.close()
            return st, eta, dec, pred
        solve()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            st, eta, dec, pred = solve()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        out[mode] = {"ms_per_solve": ms, "headline_speedup_over_this": ms / head_ms,
                     "eta": eta, "status": st}
        if mode != "off":
            out[mode]["prediction_accuracy"] = float(np.mean(pred == dec))
    return out


def config_sweep(args, params):
    """The other workloads of the method's configurations, each timed on its own (CUDA events
    around whole solves after one untimed solve), with accuracy next to the time:
      C1  N=1024, nb=128, iid N(0,1), Max alpha=100 / FORCE_LU / FORCE_QR, FP64; the threaded
          oracle's full solve of the same system timed beside it;
      C2  N=16384, nb=256, iid N(0,1), FP64: Max alpha=100 and 6000, MUMPS alpha=2.1;
      C3  N=32768, nb=256, A=U diag(s) V^T, FP32 + FP64 refinement: kappa 1e2 and 1e8 at
          alpha=100 (GMRES-IR at 1e8), and kappa 1e5 at the paper-scale alpha=6000;
      C5  N=65536, nb=512, iid N(0,1) with 10 % of the diagonal tiles scaled by 1e-8, Max
          alpha=1e5, FP32 + FP64 GMRES-IR, speculation off / repeat-previous / MLP."""
    import numpy as np
    import torch
    from oracle import luqr_oracle as O
    from oracle import luqr_oracle_mt as MT
    from paper_1401_5522_gb300 import inputs, luqr
    stream = torch.cuda.current_stream()
    out = {}

    def timed(name, A, nb, crit, alpha, prec, reps=1, refine="classic", **kw):
        N = A.shape[0]
        b = (A @ torch.ones(N, 1, dtype=torch.float64, device="cuda")).reshape(-1).contiguous()
        res = {}

        def solve():
            if prec == "fp64":
                x = b.clone()
                h = luqr.factor(A, nb, crit, alpha, b=x, tree="binary_tt", precision="fp64", **kw)
                st, its, eta = h.sync(), 0, None
            else:
                x = torch.zeros(N, dtype=torch.float64, device="cuda")
                h = luqr.factor(A, nb, crit, alpha, tree="binary_tt", precision="fp32", **kw)
                if refine == "gmres":
                    st, its, eta = h.refine_gmres(A, b, x, tol=args.tol, max_iter=20, restart=40)
                else:
                    st, its, eta = h.refine(A, b, x, tol=args.tol, max_iter=30)
            dec, _ = h.decisions()
            pred = h.features()[1] if kw.get("speculate", "off") != "off" else None
            h.close()
            res.update(status=st, iters=its, dec=dec, x=x, pred=pred)

        solve()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            solve()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        x = res["x"]
        r = b - A @ x
        nA = A.abs().sum(dim=1).max()
        eta = float(r.abs().max() / (nA * x.abs().max() + b.abs().max()))
        hpl3 = float(r.abs().max() / (nA * x.abs().max() * 2.0 ** -53 * N))
        d = {"ms_per_solve": ms, "gflops_normalized": (2.0 / 3.0) * N ** 3 / (ms / 1e3) / 1e9,
             "eta": eta, "hpl3": hpl3, "lu_fraction": float(np.mean(res["dec"] == 1)),
             "status": int(res["status"]), "ir_iters": int(res["iters"]), "timed_solves": reps}
        if res["pred"] is not None:
            d["prediction_accuracy"] = float(np.mean(res["pred"] == res["dec"]))
        out[name] = d
        return d

    # C1 with the oracle beside it
    A1 = inputs.gaussian(1024, 0, device="cuda")
    for crit, alpha in (("max", 100.0), ("force_lu", 0.0), ("force_qr", 0.0)):
        d = timed(f"C1 N=1024 nb=128 {crit} alpha={alpha:g} fp64", A1, 128, crit, alpha, "fp64",
                  reps=3)
        An = A1.cpu().numpy()
        bn = An @ np.ones(1024)
        t0 = time.perf_counter()
        xo, fo = MT.solve(An, bn, 128, {"max": O.CRIT_MAX, "force_lu": O.CRIT_FORCE_LU,
                                        "force_qr": O.CRIT_FORCE_QR}[crit], alpha, tree=1)
        to = time.perf_counter() - t0
        d["oracle"] = {"seconds": to, "threads": fo.threads, "nproc": os.cpu_count(),
                       "eta": O.backward_error(An, xo, bn),
                       "gflops_normalized": (2.0 / 3.0) * 1024 ** 3 / to / 1e9}
    del A1
    # C2 subset (FP64)
    A2 = inputs.gaussian(16384, 0, device="cuda")
    for crit, alpha in (("max", 100.0), ("max", 6000.0), ("mumps", 2.1)):
        timed(f"C2 N=16384 nb=256 {crit} alpha={alpha:g} fp64", A2, 256, crit, alpha, "fp64")
    del A2
    torch.cuda.empty_cache()
    # C3 variants
    for kappa, alpha, ref in ((1e2, 100.0, "classic"), (1e5, 6000.0, "classic")):
        A3 = inputs.conditioned(32768, kappa, seed=0, device="cuda")
        timed(f"C3 N=32768 nb=256 kappa={kappa:g} max alpha={alpha:g} fp32+{ref} IR", A3, 256,
              "max", alpha, "fp32", reps=2, refine=ref)
        del A3
        torch.cuda.empty_cache()
    # kappa = 1e8: u_fp32 kappa ~ 6, the FP32 factorization is no usable preconditioner at this
    # size (GMRES-IR stalls near eta 1e-3); the FP64 factorization is the path there
    A3 = inputs.conditioned(32768, 1e8, seed=0, device="cuda")
    timed("C3 N=32768 nb=256 kappa=1e+08 max alpha=100 fp64 factorization", A3, 256, "max",
          100.0, "fp64", reps=1)
    del A3
    torch.cuda.empty_cache()
    # C5 learned speculation
    n5 = 65536 // 512
    A5 = inputs.gaussian(65536, 5, device="cuda")
    A5 = inputs.scale_diag_tiles(A5, 512, inputs.choose_panels(n5, 0.1, 5), 1e-8)
    for mode in ("off", "repeat", "mlp"):
        kw = {"speculate": mode}
        if mode == "mlp":
            if params is None:
                continue
            kw["mlp_params"] = params
        timed(f"C5 N=65536 nb=512 max alpha=1e5 fp32+gmres IR speculate={mode}", A5, 512, "max",
              1e5, "fp32", reps=1, refine="gmres", **kw)
    del A5
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ main GPU leg
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    config = {"workload": (f"hybrid LU-QR solve, N={args.N}, nb={args.nb}, A=U diag(s) V^T "
                           f"kappa={args.kappa:g}, b=A*1, {args.criterion} alpha={args.alpha:g}, "
                           f"{tree_desc(args)}, {args.precision} factorization + FP64 refinement to "
                           f"eta<={args.tol:g}, {args.speculate} speculation"),
              "N": args.N, "nb": args.nb, "kappa": args.kappa, "criterion": args.criterion,
              "alpha": args.alpha, "tree": args.tree, "factor_precision": args.precision,
              "refinement": "fp64", "fp32_kernels": args.fp32_kernels,
              "speculate": args.speculate,
              "parallelism": f"replicas x{args.gpus}",
              "l2": "inputs larger than L2 (A is N^2 float64)"}

    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(reference_arm(args, config)))
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1401_5522_gb300 import build as B
    B.build()
    from paper_1401_5522_gb300 import inputs, luqr

    N, nb = args.N, args.nb
    A = inputs.conditioned(N, args.kappa, seed=args.seed + rank, device="cuda")
    b = (A @ torch.ones(N, 1, dtype=torch.float64, device="cuda")).reshape(-1).contiguous()
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    info = {}
    spec = {"speculate": args.speculate}
    mlp_params, train_info = (train_decision_mlp(args) if args.speculate == "mlp" or args.forms
                              else (None, None))
    if args.speculate == "mlp":
        spec["mlp_params"] = mlp_params
    policy = (args.tree, args.tree_small, args.tree_switch, args.group)
    tuning = None
    if args.tune_tree:
        from paper_1401_5522_gb300 import autotune
        policy, table = autotune.tune_tree(A, nb, args.criterion, args.alpha, args.precision,
                                           fp32_kernels=args.fp32_kernels)
        tuning = {"chosen": list(policy),
                  "factor_ms": [[list(p), round(t, 2)] for p, t in table]}
        config["tree"], config["tree_small"], config["tree_switch"], config["group"] = policy
        old_desc = tree_desc(args)
        args.tree, args.tree_small, args.tree_switch, args.group = policy
        config["workload"] = config["workload"].replace(old_desc, tree_desc(args))
    elif args.tree_switch or args.tree == "grouped":
        config["tree_small"], config["tree_switch"] = args.tree_small, args.tree_switch
        config["group"] = args.group

    def one_solve():
        h = luqr.factor(A, nb, args.criterion, args.alpha, tree=policy[0], tree_small=policy[1],
                        tree_switch=policy[2], group=policy[3], precision=args.precision,
                        fp32_kernels=args.fp32_kernels, **spec)
        st, its, eta = h.refine(A, b, x, tol=args.tol, max_iter=30)
        dec, _ = h.decisions()
        info["hpl3"] = h.accuracy()[1] if st == 0 else None     # host-side, no sync
        if args.speculate != "off":
            info["pred"] = h.features()[1]
        h.close()
        info["iters"] = its
        info["eta"] = eta
        info["status"] = st
        info["dec"] = dec
        return st

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        one_solve()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    # inside the timed region only the tensor-core update's launches carry CUDA events (the
    # others are counted): events on all ~20 000 launches of a solve cost about 3 %
    gemm_roles = sorted(l for l, f in KERNEL_OF_LABEL.items() if f == "k_gemm_tc4")
    luqr.profile(True, True)
    luqr.profile_select(gemm_roles)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    statuses, iters = [], []
    for _ in range(args.steps):
        statuses.append(one_solve())
        iters.append(info["iters"])
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    prof = luqr.profile_read()
    luqr.profile_select(None)
    luqr.profile(False, True)
    clk = clocks.stop()
    # every kernel's device time, from one more (untimed) solve: dominance and shares
    luqr.profile(True, True)
    one_solve()
    prof_all = luqr.profile_read()
    luqr.profile(False, True)
    flops = (2.0 / 3.0) * float(N) ** 3
    ms, value = job_rate(ms, world, flops, "cuda")
    eta_gpu = info["eta"]
    dec = info["dec"]
    n = len(dec)

    # ---------------- roofline of the dominant kernel (CUDA events inside the timed region)
    fac = step_kernel_flops(dec, n, nb, policy, 0, replay=False)
    rep = step_kernel_flops(dec, n, nb, policy, 0, replay=True)
    total_alg = {k: args.steps * fac.get(k, 0.0) + sum(iters) * rep.get(k, 0.0)
                 for k in set(fac) | set(rep)}
    tc_bytes = step_tc_bytes(dec, n, nb, policy, 0) if args.precision == "fp32" else {}
    # the profiler labels launches by role; the dominant kernel is the CUDA function with the
    # most device time, summed over the roles it serves
    funcs = {}
    for label, (launches, tot_ms) in prof_all.items():
        f = KERNEL_OF_LABEL.get(label, label)
        e = funcs.setdefault(f, [0, 0.0, []])
        e[0] += launches
        e[1] += tot_ms
        e[2].append(label)
    dom = max(funcs.items(), key=lambda kv: kv[1][1]) if funcs else None
    roofline = None
    all_ms1 = sum(v[1] for v in prof_all.values()) if prof_all else 0.0
    if dom is not None:
        name, (_, ms1, labels) = dom
        share = ms1 / all_ms1 if all_ms1 else None
        # launches and device time of the dominant kernel over the timed steps
        launches = sum(prof.get(l, (0, 0.0))[0] for l in labels)
        tot_ms = sum(prof.get(l, (0, 0.0))[1] for l in labels)
        if any(l in tc_bytes for l in labels) and tot_ms > 0.0:
            # algorithmic work (trailing matrix read + written once per step; Table I update
            # flops) of the bulk update over the timed steps, per the kernel's own launch time
            peaks = load_peaks()
            ub, uf = update_work(dec, n, nb, policy, 4)
            alg_bytes = args.steps * ub
            gbs = alg_bytes / (tot_ms / 1e3) / 1e9
            tf32_peak = peaks["bf16_tflops_sustained"] * TF32_PER_BF16
            mma_tflops = 3.0 * args.steps * uf / (tot_ms / 1e3) / 1e12   # 3xTF32: 3 MMAs a product
            hbm = {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                   "frac": gbs / peaks["hbm_gbs"],
                   "peak_source": f"{peaks['source']} HBM copy bandwidth"}
            ten = {"achieved": mma_tflops, "peak": tf32_peak, "unit": "TFLOP/s",
                   "frac": mma_tflops / tf32_peak,
                   "peak_source": (f"{peaks['source']} sustained BF16 cuBLAS x 1.1/2.25 "
                                   "(nominal dense TF32/BF16 ratio); achieved counts the 3 TF32 "
                                   "MMAs of each 3xTF32 product of the Table I update flops")}
            main, other = (("hbm", hbm), ("tensor", ten)) if hbm["frac"] >= ten["frac"] else \
                (("tensor", ten), ("hbm", hbm))
            pass_bytes = args.steps * sum(tc_bytes.get(l, 0.0) for l in labels)
            roofline = {"bound": main[0], "kernel": name, "roles": labels, **main[1],
                        "traffic": traffic_per_launch(name, alg_bytes / launches),
                        "other_roof": {"bound": other[0], **other[1]},
                        "bytes_per_launch": alg_bytes / launches,
                        "flops_per_launch": args.steps * uf / launches,
                        "pass_model_bytes_per_launch": pass_bytes / launches,
                        "launches": launches, "avg_launch_ms": tot_ms / launches,
                        "share_of_kernel_time": share,
                        "timing": "CUDA events on the kernel's launches over the timed steps"}
        else:
            # not timed inside the timed region: the extra profiled solve's durations
            launches = sum(prof_all.get(l, (0, 0.0))[0] for l in labels)
            tot_ms = sum(prof_all.get(l, (0, 0.0))[1] for l in labels)
            total_alg = {k: fac.get(k, 0.0) + info["iters"] * rep.get(k, 0.0)
                         for k in set(fac) | set(rep)}
            alg = sum(total_alg.get(l, 0.0) for l in labels)
            peak = FP32_FFMA_PEAK_TFLOPS if args.precision == "fp32" else FP64_DFMA_PEAK_TFLOPS
            if alg:
                achieved = alg / (tot_ms / 1e3) / 1e12
                roofline = {"bound": "alu", "kernel": name, "roles": labels,
                            "achieved": achieved, "peak": peak,
                            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                            "peak_source": ("derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"
                                            if args.precision == "fp32" else
                                            "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz"),
                            "launches": launches, "avg_launch_ms": tot_ms / launches,
                            "share_of_kernel_time": share,
                            "timing": "CUDA events of one extra profiled solve"}
    gpu_launches = int(sum(v[0] for v in prof.values())) if prof else 0
    kernel_table = {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in
                    sorted(prof_all.items(), key=lambda kv: -kv[1][1])}

    # ---------------- end to end through the C interface with host buffers
    e2e = None
    if args.e2e_steps > 0:
        hA = torch.empty((N, N), dtype=torch.float64, pin_memory=True).t()
        hA.copy_(A)
        hb = torch.empty(N, dtype=torch.float64, pin_memory=True)
        hb.copy_(b)
        hx = torch.empty(N, dtype=torch.float64, pin_memory=True)
        dA2 = torch.empty_like(A)
        db2 = torch.empty_like(b)
        dx2 = torch.empty_like(x)
        torch.cuda.synchronize()
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.e2e_steps):
            dA2.copy_(hA, non_blocking=True)
            db2.copy_(hb, non_blocking=True)
            h = luqr.factor(dA2, nb, args.criterion, args.alpha, **tree_kw(args),
                            precision=args.precision, fp32_kernels=args.fp32_kernels, **spec)
            h.refine(dA2, db2, dx2, tol=args.tol, max_iter=30)
            h.close()
            hx.copy_(dx2, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = f0.elapsed_time(f1) / args.e2e_steps
        e2e = {"value": flops * world / (e2e_ms / 1e3) / 1e9, "unit": "GFLOP/s",
               "ms_per_step": e2e_ms, "h2d_bytes_per_step": 8 * N * N + 8 * N,
               "d2h_bytes_per_step": 8 * N}
        del hA, dA2

    # ---------------- plain FP64 GPU solve (the denominator), one timed solve
    plain = None
    if args.fp64_baseline:
        small = inputs.conditioned(1024, args.kappa, seed=1, device="cuda")
        sb = (small @ torch.ones(1024, 1, dtype=torch.float64, device="cuda")).reshape(-1).contiguous()
        luqr.factor(small, nb, args.criterion, args.alpha, b=sb, **tree_kw(args),
                    precision="fp64").close()                    # loads the FP64 kernels
        times = []
        for _ in range(args.fp64_baseline):
            bb = b.clone()
            torch.cuda.synchronize()
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            h = luqr.factor(A, nb, args.criterion, args.alpha, b=bb, **tree_kw(args),
                            precision="fp64")
            g1.record(stream)
            torch.cuda.synchronize()
            st64, _, _ = h.info()
            dec64, _ = h.decisions()
            h.close()
            times.append(g0.elapsed_time(g1))
        p_ms = statistics.median(times)
        r = b - A @ bb
        eta64 = float(r.abs().max() / (A.abs().sum(dim=1).max() * bb.abs().max() + b.abs().max()))
        plain = {"ms_per_solve": p_ms, "ms_each": times, "timed_solves": len(times),
                 "gflops": flops / (p_ms / 1e3) / 1e9, "eta": eta64,
                 "status": st64, "decisions_equal_to_fp32_path": bool(np.array_equal(dec64, dec)),
                 "speedup_of_headline": p_ms / ms}

    forms = None
    if args.forms:
        forms = {"speculation": speculation_form(args, A, b, x, ms, mlp_params, train_info),
                 "batched": batched_form(args)}
        if plain is not None:
            for key in ("off", "repeat", "mlp"):
                if key in forms["speculation"]:
                    forms["speculation"][key]["speedup_vs_plain_fp64"] = (
                        plain["ms_per_solve"] / forms["speculation"][key]["ms_per_solve"])

    sweep = None
    if args.configs and world == 1:
        sweep = config_sweep(args, mlp_params)
    if rank != 0:
        return
    try:
        cpu = oracle_sample(A.cpu().numpy(), args, steps=args.cpu_steps)
    except Exception as exc:       # the baseline is context; keep the GPU line
        cpu = {"error": repr(exc)[-300:]}
    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic", "config": config,
            "eta": eta_gpu, "hpl3": info.get("hpl3"), "hpl3_eps": "2^-53",
            "ir_iters": iters, "status": statuses,
            "lu_fraction": float(np.mean(dec == 1)),
            "speculation": {"mode": args.speculate,
                            "prediction_accuracy": (float(np.mean(info["pred"] == dec))
                                                    if "pred" in info else None)},
            "plain_fp64": plain, "roofline": roofline, "gpu_launches": gpu_launches,
            "kernels": kernel_table, "kernels_scope": "one extra profiled solve (all kernels timed)",
            "e2e": e2e, "clocks": clk, "forms": forms, "configs": sweep, "tree_tuning": tuning,
            "cpu_baseline": cpu_baseline_dict(cpu, args)}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
