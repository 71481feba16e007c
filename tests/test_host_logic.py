"""Host-side logic of the Python package that needs no GPU: folding the feature
standardisation into the MLP's first layer, the repeat-previous predictor, and the batched
solver's size buckets."""
import os
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_1401_5522_gb300 import batched as Bt
from paper_1401_5522_gb300 import speculation as S


def test_folded_parameters_take_raw_features():
    rng = np.random.default_rng(0)
    p = S.init_params(3).astype(np.float64)
    p[1024:1088] = 0.1 * rng.standard_normal(64)          # nonzero first-layer biases
    X = rng.standard_normal((50, 16)) * 5.0 + 2.0
    mu = X.mean(axis=0)
    sigma = X.std(axis=0)
    folded = S.fold_standardisation(p, mu, sigma).astype(np.float64)
    want = M.forward(p, (X - mu) / sigma)
    got = M.forward(folded, X)
    assert np.max(np.abs(got - want)) <= 1e-5 * max(1.0, np.max(np.abs(want)))


def test_init_params_layout():
    p = S.init_params(0)
    assert p.shape == (M.NPARAMS,) and p.dtype == np.float32
    assert np.all(p[1024:1088] == 0) and p[-1] == 0          # zero biases


def test_repeat_previous():
    out = S.repeat_previous([[0, 1, 1, 0], []])
    assert out[0].tolist() == [1.0, 0.0, 1.0, 1.0]
    assert len(out[1]) == 0


def test_size_buckets_cover_every_size_once():
    seen = [Bt.bucket_of(N) for N in range(1, 2049)]
    assert min(seen) == 0 and max(seen) == len(Bt.BUCKETS) - 1
    assert all(a <= b for a, b in zip(seen, seen[1:]))      # monotone in N
    for i, (lo, hi) in enumerate(Bt.BUCKETS):
        assert Bt.bucket_of(lo) == i and Bt.bucket_of(hi) == i
    table = {0: 32, 3: 64}
    assert Bt.nb_for([Bt.BUCKETS[0][0], Bt.BUCKETS[3][1], Bt.BUCKETS[1][0]], table, 48) == [32, 64, 48]


def test_bench_defaults_follow_the_measurement_contract():
    import bench
    a = bench.parse([])
    assert a.gpus == 1 and a.impl == "luqr"
    assert a.warmup >= 3 and a.steps >= 1
    assert (a.N, a.nb, a.kappa, a.criterion, a.alpha) == (32768, 256, 1e5, "max", 100.0)
    # the tree policy whose full-size decisions are stored (tests/golden/large_c3p_*.json)
    assert (a.tree, a.tree_small, a.tree_switch, a.group) == ("grouped", "binary_tt", 64, 4)
    assert a.tol == 1e-13 and a.e2e_steps >= 1


def test_bench_update_work_follows_the_trailing_matrix_model():
    """Bytes of the bulk update = trailing rows k.. x bulk columns read + written once per
    step; summed over a run they approach (2/3) s_C N^3 / nb, the per-solve algorithmic
    bytes of the trailing update; flops approach Table I's update terms."""
    import numpy as np
    import bench
    n, nb = 128, 256
    N = n * nb
    qr = np.zeros(n, dtype=np.uint8)
    qr[-1] = 1
    by, fl = bench.update_work(qr, n, nb, "binary_tt", 4)
    m = np.arange(n - 1, -1, -1, dtype=float)           # m = n-1-k
    cols = np.maximum(m - 1, 0) * nb
    assert by == pytest.approx(float(np.sum(8.0 * (m + 1) * nb * cols)))
    assert by == pytest.approx((2.0 / 3.0) * 4 * N ** 3 / nb, rel=0.03)
    # all-QR update flops ~ 4/3 N^3 (UNMQR + TTMQR on every trailing tile) up to O(N^2 nb)
    assert fl == pytest.approx((4.0 / 3.0) * N ** 3, rel=0.03)
    lu = np.ones(n, dtype=np.uint8)
    _, fl_lu = bench.update_work(lu, n, nb, "binary_tt", 4)
    assert fl_lu == pytest.approx((2.0 / 3.0) * N ** 3, rel=0.03)


def test_tree_autotuner_candidates():
    from paper_1401_5522_gb300 import autotune
    c = autotune.candidates(128)
    assert ("binary_tt", "binary_tt", 0, 4) in c and ("grouped", "binary_tt", 0, 8) in c
    assert ("grouped", "binary_tt", 64, 4) in c and ("binary_tt", "grouped", 96, 8) in c
    assert all(t != s for t, s, w, g in c if w > 0)
    assert all(g == 4 for t, s, w, g in c if "grouped" not in (t, s))
    assert len(set(c)) == len(c)
    assert {w for _, _, w, _ in autotune.candidates(4)} == {0, 2, 3}


def test_bench_tree_counts_cover_every_tile():
    """(singles, TS, TT) of each tree: every sub-diagonal tile is killed exactly once and each
    GEQRT single is a tile that is later an eliminator or tile k (singles - 1 = TT kills)."""
    import bench
    for m in range(0, 40):
        for pol in ("flat_ts", "binary_tt", ("grouped", "grouped", 0, 3), ("grouped", "x", 0, 8)):
            s, ts, tt = bench.tree_counts(pol, m)
            assert ts + tt == m and s >= 1
            if bench.tree_at(pol, m) != "flat_ts":
                assert s - 1 == tt
    assert bench.tree_at(("grouped", "binary_tt", 16, 4), 15) == "binary_tt"
    assert bench.tree_at(("grouped", "binary_tt", 16, 4), 16) == "grouped"


SMEM_RECORD_CHECK = r"""
#include <cassert>
#include <cstdio>
#include <thread>
#include <vector>
#include "smem_record.h"
int main() {
  luqr::SmemRecord rec;
  int calls = 0;
  auto ok = [&](size_t) { ++calls; return true; };
  auto bad = [&](size_t) { ++calls; return false; };
  assert(rec.ensure(0, 40 * 1024, ok) && calls == 0);        // below the default
  assert(rec.ensure(0, 100 * 1024, ok) && calls == 1);       // raised on device 0
  assert(rec.ensure(0, 100 * 1024, ok) && calls == 1);       // recorded
  assert(rec.ensure(0, 64 * 1024, ok) && calls == 1);        // below the record
  assert(rec.ensure(1, 100 * 1024, ok) && calls == 2);       // device 1 has its own record
  assert(!rec.ensure(2, 200 * 1024, bad) && calls == 3);     // a failed raise is not recorded
  assert(rec.ensure(2, 200 * 1024, ok) && calls == 4);
  assert(rec.ensure(99, 100 * 1024, ok) && calls == 5);      // beyond the table: every time
  assert(rec.ensure(99, 100 * 1024, ok) && calls == 6);
  assert(rec.ensure(-1, 40 * 1024, ok) && calls == 6);
  // many host threads on one device: the attribute is set once
  luqr::SmemRecord r2;
  int n = 0;
  std::vector<std::thread> th;
  for (int t = 0; t < 16; ++t)
    th.emplace_back([&] { for (int i = 0; i < 1000; ++i) r2.ensure(3, 120 * 1024, [&](size_t) { ++n; return true; }); });
  for (auto& x : th) x.join();
  assert(n == 1);
  std::puts("ok");
  return 0;
}
"""


def test_dynamic_smem_record_is_per_device(tmp_path):
    """The record behind ensure_dyn_smem (csrc/smem_record.h) keeps one limit per device,
    records only successful raises, and sets the attribute once under concurrent callers."""
    import shutil
    import subprocess
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    src = tmp_path / "check.cpp"
    src.write_text(SMEM_RECORD_CHECK)
    exe = tmp_path / "check"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_1401_5522_gb300", "csrc")
    subprocess.run([gxx, "-std=c++17", "-O1", "-pthread", "-I", inc, str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True)
    assert out.stdout.strip() == "ok"
