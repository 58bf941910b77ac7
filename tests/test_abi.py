"""The C-ABI library loads and exports every entry point include/mb.h declares
(no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(mb_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for want in ("mb_render", "mb_version", "mb_strerror", "mb_fp64_peak"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2007_00745_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls_work_without_gpu():
    import paper_2007_00745_gb300 as mb
    assert mb.mb_version().startswith("mb ")
    assert mb.mb_strerror(1) == "invalid argument"
    assert mb.mb_strerror(99) == "unknown error"


def test_missing_library_fails_loudly(tmp_path):
    """Without libmb.so the first call raises ImportError: no CPU fallback."""
    import shutil
    import subprocess
    import sys
    pkg = os.path.join(ROOT, "paper_2007_00745_gb300")
    dst = tmp_path / "paper_2007_00745_gb300"
    dst.mkdir()
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            shutil.copy(os.path.join(pkg, f), dst / f)
    code = ("import sys; sys.path.insert(0, %r); import paper_2007_00745_gb300 as mb; "
            "mb.mb_render((-2.0, 1.0, -1.0, 1.0), 4, 4, 10, 4.0, 0)") % str(tmp_path)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "libmb.so not built" in r.stderr
