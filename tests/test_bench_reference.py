"""bench.py --impl reference (the oracle timed on the host cores) prints one
JSON line with the contract's keys.  Runs on the CPU, on a small view."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2", "--warmup", "1",
           "--size", "256", "--iter-max", "500"]
    out = subprocess.run(cmd, check=True, capture_output=True, text=True, timeout=300, cwd=ROOT).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "Giter/s" and d["unit"] == "Giter/s"
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "Giter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "256x256" in d["config"]["workload"] and "iterMax 500" in d["config"]["workload"]
    # the same config dict our arm prints, and the same row sample as our cpu_baseline
    assert set(d["config"]) == {"workload", "l2", "parallelism", "bit_exact"}
    assert "every 4-th" in d["cpu_baseline"]["sample"]


def test_reference_arm_under_torchrun_prints_once():
    """Launched as the benchmark's N>1 command (torchrun, 2 ranks): rank 0 alone
    times the oracle and prints the line; the other rank exits 0 without work."""
    with socket.socket() as sk:          # a free port for the rendezvous
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--size", "128",
           "--iter-max", "200"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
