"""Host-side parts of bench.py (no GPU): the bounded CPU-baseline sample, the serving pool and the clock record."""
import sys
import os

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
import graphgen as gg  # noqa: E402
import oracle  # noqa: E402


class _Sized:
    def __init__(self, nnz):
        self.nnz = nnz


def test_oracle_sample_is_bounded():
    # small graphs: a full run; large ones: pass 0, iterations capped so that
    # the scanned entries stay within the sample's budget
    assert bench.oracle_sample_plan(_Sized(137_000))[:2] == (10, 20)
    for nnz in (60_000_000, 128_307_544, 900_000_000, 5_000_000_000):
        passes, iters, what = bench.oracle_sample_plan(_Sized(nnz))
        assert passes == 1 and 1 <= iters <= 20 and "pass 0" in what
        assert iters == 1 or iters * nnz <= bench.ORACLE_SAMPLE_ENTRIES


def test_oracle_sample_counts_scanned_entries():
    # prune off: every iteration of a pass scans every entry of that pass's graph
    g = gg.sbm(7, 400, 4, 0.2, 0.01)
    e, dt, q = bench.run_oracle_sample(g, oracle.SYNC, max_passes=1, max_iterations=3)
    r = oracle.louvain(g.off, g.col, g.w, mode=oracle.SYNC, prune=0, max_passes=1, max_iterations=3)
    assert e == g.nnz * r.passes[0].iterations and dt >= 0 and q == r.Q


def test_serving_pool_is_seeded_and_in_range():
    a = bench.serving_pool(bench.SEED + 4, 6, 1000, 20000)
    b = bench.serving_pool(bench.SEED + 4, 6, 1000, 20000)
    assert len(a) == 6
    for g, h in zip(a, b):
        assert g.n == h.n and (g.off == h.off).all() and (g.col == h.col).all() and (g.w == h.w).all()
        assert 1000 <= g.n <= 20000 and g.nnz > 0
        assert g.w.min() >= 1 and g.w.max() <= 8
        # symmetric: the multiset of (u, v, w) equals that of (v, u, w)
        rows = (g.off[1:] - g.off[:-1])
        u = gg_rows(rows)
        fwd = sorted(zip(u.tolist(), g.col.tolist(), g.w.tolist()))
        bwd = sorted(zip(g.col.tolist(), u.tolist(), g.w.tolist()))
        assert fwd == bwd


def gg_rows(rows):
    import numpy as np
    return np.repeat(np.arange(len(rows), dtype=np.int64), rows)


def test_oracle_baseline_runs_on_one_pinned_core_and_restores_affinity():
    import os
    import bench
    before = os.sched_getaffinity(0)
    with bench.OneCore() as pin:
        assert os.sched_getaffinity(0) == {pin.core}
        assert pin.core in before
    assert os.sched_getaffinity(0) == before


def test_clock_samples_give_median_max_and_throttle_reasons(tmp_path):
    """The clock record of the timed region: median SM clock under load, the
    maximum, and every throttle reason seen active in any sample (the sampler
    writes nvidia-smi's CSV; a malformed line is skipped)."""
    ck = bench.Clocks(0)
    ck.path = str(tmp_path / "clocks.csv")
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070",
        "0, 1500, 2070, 1000.0, 0x8, Active, Not Active, Not Active, Not Active",
    ]
    with open(ck.path, "w") as f:
        f.write("\n".join(rows) + "\n")

    class _Done:   # the sampler process has already ended
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    ck.proc = _Done()
    got = ck.stop()
    assert got["samples"] == 4
    assert got["sm_mhz"] == 2025.0 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert not os.path.exists(ck.path)


def test_clocks_without_nvidia_smi_say_so():
    ck = bench.Clocks(0)
    ck.proc = None
    got = ck.stop()
    assert got["sm_mhz"] is None and got["reasons"] == ["nvidia-smi unavailable"]
