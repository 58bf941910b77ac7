"""bench.py's own arm, end to end on a small view: one JSON line carrying every
key of the benchmark contract (throughput, roofline of the main render kernel,
the oracle's CPU baseline, the end-to-end figure, clocks and launch count),
with values that agree with one another."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_json_line_contract():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "2", "--warmup", "3", "--size", "1024",
           "--iter-max", "2000", "--no-compare", "--no-batch", "--no-serve", "--no-precision", "--no-cycle", "--no-zoom"]
    out = subprocess.run(cmd, check=True, capture_output=True, text=True, timeout=600, cwd=ROOT).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["metric"] == "Giter/s" and d["unit"] == "Giter/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 3 and d["scaling"] == "strong"
    assert d["vs_baseline"] is None and d["dtype"] == "f64" and d["data"] == "synthetic"
    c = d["config"]
    assert "1024x1024" in c["workload"] and "iterMax 2000" in c["workload"] and "learned FCFS" in c["workload"]
    assert "4 MB per step <= 129 MB L2" in c["l2"]
    # value = iterations per step / time per step
    assert d["value"] == pytest.approx(d["iterations_per_step"] / d["ms_per_step"] / 1e6, rel=1e-6)
    r = d["roofline"]
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["peak"] > 0 and r["achieved"] > 0
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-9)
    assert 0.05 < r["frac"] < 1.2
    assert r["traffic"] is None or r["traffic"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["unit"] == "Giter/s" and cb["value"] > 0 and cb["cores"] >= 1
    assert cb["sample"]
    e = d["e2e"]
    assert e["unit"] == "Giter/s" and e["value"] > 0 and e["h2d_bytes_per_step"] == 0
    assert e["d2h_bytes_per_step"] == 1024 * 1024 * 4
    ev = d["e2e_variants"]
    assert ev["direct_to_host"]["same_counts"] is True          # host-written counts equal the device render's
    assert e in (ev["direct_to_host"], ev["device_then_copy"])
    cl = d["clocks"]
    assert cl["sm_max_mhz"] > 0 and isinstance(cl["reasons"], list)
    assert d["gpu_launches"] >= 2 * d["steps"]
