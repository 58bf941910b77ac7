"""Host-side arithmetic of the benchmark: makespan and idle tail from per-CTA
trace records, and percentiles."""
import numpy as np

import bench


def _trace(rows):
    tr = np.zeros((len(rows), 3), np.int64)
    for k, (s, e, sm) in enumerate(rows):
        tr[k] = (s, e, sm)
    return tr


def test_trace_stats_idle_tail():
    # two SMs, makespan 100 ns: SM 0 ends at 100, SM 1 at 60 -> idle tail (0 + 40) / (2 * 100)
    st = bench.trace_stats(_trace([(0, 100, 0), (10, 60, 1), (0, 50, 1)]), 2)
    assert st["makespan_ms"] == 100 / 1e6
    assert st["idle_tail"] == 0.2


def test_trace_stats_ignores_unwritten_records_and_missing_sms():
    st = bench.trace_stats(_trace([(5, 105, 0), (0, 0, 0)]), 2)
    assert st["makespan_ms"] == 100 / 1e6
    assert st["idle_tail"] == 0.5     # SM 1 never ran anything


def test_percentiles():
    xs = list(range(1, 101))
    assert bench.pct(xs, 50) in (50, 51)
    assert bench.pct(xs, 99) == 99 or bench.pct(xs, 99) == 100
    assert bench.pct([], 50) is None


def test_roofline_entry_arithmetic():
    # 1.2e11 steps in 600 ms against a 0.5 T ops/s FP64 pipe: 2.5 FP64-pipe additions per step
    # on average -> 2.5 x 1.2e11 / 0.6 = 0.5e12 -> the pipe is full
    r = bench.roofline_entry(120_000_000_000, 600.0, 0.5e12, None)
    assert abs(r["fp64_pipe_frac"] - 1.0) < 1e-12
    assert r["fp64_pipe_frac_issued"] is None
    # 2.56 FP64 instructions issued per step (idle lanes, replays) on the same launch
    r2 = bench.roofline_entry(120_000_000_000, 600.0, 0.5e12, None, 2.56)
    assert abs(r2["fp64_pipe_frac_issued"] - 2.56 / 2.5) < 1e-12
    assert abs(r["frac"] - r["fp64_pipe_frac"]) < 1e-12
    assert abs(r["peak"] - 0.5 * 8 / 2.5) < 1e-12
    assert abs(r["achieved"] - 8 * 1.2e11 / 0.6 / 1e12) < 1e-12
    assert abs(r["nominal_frac"] - 8 / 2.5 * r["frac"]) < 1e-12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["traffic"] is None


def test_roofline_dram_context(monkeypatch):
    monkeypatch.setattr(bench, "measured_hbm_gbs", lambda: 5000.0)
    r = bench.roofline_entry(1000, 500.0, 1e12, 2.5e8)   # 250 MB in 0.5 s = 0.5 GB/s
    assert abs(r["dram_gbs"] - 0.5) < 1e-12 and abs(r["dram_frac_of_measured_hbm"] - 1e-4) < 1e-15
    assert bench.roofline_entry(1000, 500.0, 1e12, None)["dram_gbs"] is None


def test_spearman():
    import numpy as np
    a = np.array([1.0, 2.0, 3.0, 4.0])
    assert abs(bench.spearman(a, a * 10) - 1.0) < 1e-12
    assert abs(bench.spearman(a, -a) + 1.0) < 1e-12
    assert abs(bench.spearman(a, np.array([2.0, 1.0, 4.0, 3.0])) - 0.6) < 1e-12


def test_view_overrides_and_workload_label(monkeypatch):
    import sys
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    v = bench.bench_view(a)
    assert (v.m, v.n, v.iter_max, v.window) == (8192, 8192, 10000, (-2.0, 1.0, -1.5, 1.5))
    assert bench.bench_config(a, v, 1)["workload"].startswith("8192x8192 re[-2,1] im[-1.5,1.5] iterMax 10000")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--window=-0.2,-0.1,0.05,0.15", "--size", "4096",
                                      "--iter-max", "2000", "--sched", "fcfs_tiles", "--tile", "16"])
    a = bench.parse()
    v = bench.bench_view(a)
    assert (v.m, v.n, v.iter_max, v.window) == (4096, 4096, 2000, (-0.2, -0.1, 0.05, 0.15))
    assert "re[-0.2,-0.1] im[0.05,0.15] iterMax 2000" in bench.bench_config(a, v, 1)["workload"]
    monkeypatch.setattr(sys, "argv", ["bench.py", "--window=1,0,0,1"])
    a = bench.parse()
    try:
        bench.bench_view(a)
    except SystemExit:
        pass
    else:
        raise AssertionError("an empty window must be refused")
