"""Compile the C oracle into oracle/_build/libmb_oracle.so.

Test infrastructure only: the oracle is a plain, slow CPU restatement of the
escape-time method used to check the CUDA path; the product never loads it.
-ffp-contract=off keeps every multiply and add a separately rounded binary64
operation on both x86-64 and aarch64.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "mb_oracle.c"), os.path.join(HERE, "mb_oracle_lowp.c")]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmb_oracle.so")

FLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fno-unsafe-math-optimizations",
         "-fopenmp", "-shared", "-fPIC", "-std=c99"]


def build(force: bool = False) -> str:
    """Build the oracle library if missing or stale; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in SRCS)):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc"] + FLAGS + ["-o", tmp] + SRCS + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
