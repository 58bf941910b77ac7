"""The command-line renderer (python -m paper_2007_00745_gb300): arguments on
the CPU; on the GPU, the written PPM equals the oracle's counts coloured by the
oracle's palette, byte for byte."""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_cli_arguments():
    from paper_2007_00745_gb300 import __main__ as cli
    a = cli.make_parser().parse_args(["--size", "48x64", "--window", "-2", "1", "-1", "1", "--sched", "naive"])
    assert a.size == (48, 64) and a.window == [-2.0, 1.0, -1.0, 1.0] and a.sched == "naive"
    with pytest.raises(SystemExit):
        cli.make_parser().parse_args(["--size", "48"])
    out = subprocess.run([sys.executable, "-m", "paper_2007_00745_gb300", "--help"], cwd=ROOT,
                         capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and "--escape-radius" in out.stdout


def _read_ppm(path):
    with open(path, "rb") as f:
        data = f.read()
    parts = data.split(b"\n", 3)
    assert parts[0] == b"P6"
    n, m = map(int, parts[1].split())
    assert parts[2] == b"255"
    return m, n, np.frombuffer(parts[3], np.uint8).reshape(m, n, 3)


@pytest.mark.gpu
@pytest.mark.parametrize("extra", [[], ["--sched", "learned", "--tile", "32"], ["--cycle-check"]])
def test_cli_writes_the_oracle_image(orc, extra):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "m.ppm")
        cmd = [sys.executable, "-m", "paper_2007_00745_gb300", "--size", "60x80", "--iter-max", "300",
               "--window", "-2", "1", "-1", "1", "--out", path] + extra
        r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr
        assert "computational process time" in r.stdout and "total process time" in r.stdout
        m, n, img = _read_ppm(path)
    assert (m, n) == (60, 80)
    want = orc.colorize(orc.render((-2.0, 1.0, -1.0, 1.0), 60, 80, 300, 4.0), 300).reshape(60, 80, 3)
    assert np.array_equal(img, want)
