"""Launch profiler: per-kernel counts and the trace-mode timeline of one factorization."""
import numpy as np
import pytest

from paper_1401_5522_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1401_5522_gb300 import build
    build.build()


def test_profile_counts_and_trace_agree():
    from paper_1401_5522_gb300 import luqr
    A = inputs.gaussian(1024, 3, device="cuda")
    luqr.profile(True, True, trace=True)
    try:
        h = luqr.factor(A, 128, "max", 100.0, precision="fp32")
        h.sync()
        h.close()
        counts = luqr.profile_read()
        trace = luqr.profile_trace()
    finally:
        luqr.profile(False, True)
    assert sum(c for c, _ in counts.values()) == len(trace)
    names = {t[0] for t in trace}
    assert names == set(counts)
    assert {"k_panel_stats", "k_getrf", "k_decide"} <= names
    t0 = np.array([t[1] for t in trace])
    t1 = np.array([t[2] for t in trace])
    assert np.all(t1 >= t0) and np.all(t0 >= 0.0)
    # per-kernel totals equal the sums of the timeline's durations
    for name, (_, ms) in counts.items():
        tot = sum(t[2] - t[1] for t in trace if t[0] == name)
        assert abs(tot - ms) <= 1e-3 * max(1.0, ms)
    # the panel stream runs one statistics launch per step, in step order
    stats = [t for t in trace if t[0] == "k_panel_stats"]
    assert len(stats) == 1024 // 128
    assert len({t[3] for t in stats}) == 1
    assert all(a[1] <= b[1] for a, b in zip(stats, stats[1:]))


def test_profile_rejects_bad_mode():
    from paper_1401_5522_gb300 import luqr
    assert luqr.lib().luqr_profile(3, 0) == luqr.ERR_INVALID


def test_profile_select_times_only_named_kernels():
    from paper_1401_5522_gb300 import luqr
    A = inputs.gaussian(512, 4, device="cuda")
    luqr.profile(True, True)
    try:
        luqr.profile_select(["k_getrf"])
        h = luqr.factor(A, 64, "max", 100.0)
        h.sync()
        h.close()
        sel = luqr.profile_read()
    finally:
        luqr.profile_select(None)
        luqr.profile(False, True)
    assert sel["k_getrf"][0] == 512 // 64 and sel["k_getrf"][1] > 0.0
    others = {k: v for k, v in sel.items() if k != "k_getrf"}
    assert others and all(v[0] > 0 and v[1] == 0.0 for v in others.values())
