"""Elimination-tree autotuner for the single-system solver.

Sec. II-C leaves the elimination list of a QR step free (any order of TS/TT kills that
zeroes the panel is valid), and Sec. IV-B builds its trees from a flat and a binary part.
The library takes a per-step policy: `tree` while a step has at least `tree_switch`
sub-diagonal tiles, `tree_small` below that.  Which policy is fastest depends on the
machine, the tile size and the number of tiles, so this module times candidate policies on
the GPU and returns the fastest.

The tree changes more than the speed.  A QR step's R block is unique up to row signs, but the
rows below it are the trailing matrix multiplied by an orthogonal factor that depends on the
tree, and the per-tile norms the criteria read are not invariant under it: two policies can
take different decisions on the same matrix (both correct runs of the method).  The tuner
therefore times the caller's own criterion on the caller's matrix (or a probe drawn from the
same recipe), and each policy has its own oracle run to be checked against.

Marshalling and timing only: every factorization runs in libluqr.so.
"""
from __future__ import annotations

import itertools

import torch

from . import luqr

TREE_NAMES = ("flat_ts", "binary_tt", "grouped")


def candidates(n_tiles, trees=("binary_tt", "grouped"), small=("binary_tt", "grouped"),
               switches=None, groups=(2, 4, 8)):
    """Candidate policies (tree, tree_small, tree_switch, group) for a matrix of n_tiles tile
    rows: every big tree alone, and every (big, small) pair with the switch at 1/8, 1/4, 1/2
    and 3/4 of the tile count (at least 2 tiles); the grouped tree with groups of each size
    in `groups`."""
    if switches is None:
        switches = sorted({max(2, (n_tiles * f) // 8) for f in (1, 2, 4, 6)})
    out = []
    for t, s, w in [(t, "binary_tt", 0) for t in trees] + \
            [(t, s, int(w)) for t, s, w in itertools.product(trees, small, switches) if s != t]:
        uses_group = "grouped" in (t, s if w else t)
        for g in (groups if uses_group else (4,)):   # the group size is unused there
            out.append((t, s, w, g))
    return out


def time_policy(A, nb, criterion, alpha, policy, precision="fp64", reps=1, **factor_kw):
    """Median device time (ms) of `reps` factorizations of A under one policy (the solver
    reads A and factors a copy of its own, so every repetition sees the same matrix)."""
    tree, small, switch, group = policy
    stream = torch.cuda.current_stream()
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        h = luqr.factor(A, nb, criterion, alpha, tree=tree, tree_small=small,
                        tree_switch=switch, group=group, precision=precision, **factor_kw)
        st = h.sync()
        e1.record(stream)
        torch.cuda.synchronize()
        h.close()
        if st != luqr.OK:
            raise luqr.LuqrError(st, "factor during tuning")
        times.append(e0.elapsed_time(e1))
    times.sort()
    return times[len(times) // 2]


def tune_tree(A, nb, criterion="max", alpha=100.0, precision="fp64", reps=1, policies=None,
              warmup=1, **factor_kw):
    """Time every candidate policy on A (a column-major float64 CUDA matrix) and return
    (best_policy, table), table a list of (policy, ms) in candidate order.  The tuned policy
    p is used as luqr.factor(..., tree=p[0], tree_small=p[1], tree_switch=p[2], group=p[3])."""
    luqr._check_matrix(A)
    n_tiles = (A.shape[0] + nb - 1) // nb
    pols = list(policies) if policies is not None else candidates(n_tiles)
    for _ in range(warmup):
        time_policy(A, nb, criterion, alpha, pols[0], precision, 1, **factor_kw)
    table = [(p, time_policy(A, nb, criterion, alpha, p, precision, reps, **factor_kw))
             for p in pols]
    best = min(table, key=lambda pm: pm[1])[0]
    return best, table
