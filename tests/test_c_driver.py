"""The C ABI without Python: tests/c_abi_driver.c is compiled with gcc against
include/mb.h and linked with libmb.so (and, as test infrastructure, the
oracle library).  On the CPU it must build and link; on the GPU it must run
and find every image equal to the oracle's."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _build(outdir):
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    from oracle import build as obuild
    from paper_2007_00745_gb300 import build as mbuild
    lib = os.path.dirname(mbuild.build())
    olib = os.path.dirname(obuild.build())
    exe = os.path.join(outdir, "c_abi_driver")
    cudalib = os.path.join(CUDA, "lib64")
    cmd = ["gcc", "-std=c99", "-O1", "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           os.path.join(ROOT, "tests", "c_abi_driver.c"), "-o", exe,
           "-L", lib, "-lmb", "-L", olib, "-lmb_oracle", "-L", cudalib, "-lcudart",
           "-Wl,-rpath," + lib, "-Wl,-rpath," + olib, "-Wl,-rpath," + cudalib]
    subprocess.run(cmd, check=True)
    return exe


def test_c_driver_builds_and_links():
    if not os.path.isdir(os.path.join(CUDA, "include")):
        pytest.skip("needs the CUDA toolkit headers")
    with tempfile.TemporaryDirectory() as d:
        assert os.path.exists(_build(d))


@pytest.mark.gpu
def test_c_driver_runs_on_the_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    with tempfile.TemporaryDirectory() as d:
        exe = _build(d)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    assert "c driver ok" in r.stdout
