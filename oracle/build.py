"""Builds the oracle's shared library (``oracle/_build/liboracle.so``) with gcc.

The oracle is test infrastructure: plain FP64 C compiled without floating-point
contraction (``-ffp-contract=off``) so that its Gaussian transform is a fixed
sequence of correctly rounded IEEE-754 operations.  OpenMP is used when the
compiler supports it; results do not depend on the thread count.
"""
from __future__ import annotations

import os
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def _openmp_flag(cc: str) -> list[str]:
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        with open(src, "w") as f:
            f.write("#include <omp.h>\nint main(void){return omp_get_max_threads() > 0 ? 0 : 1;}\n")
        r = subprocess.run([cc, "-fopenmp", src, "-o", os.path.join(d, "t")],
                           capture_output=True)
        return ["-fopenmp"] if r.returncode == 0 else []


def build(force: bool = False) -> str:
    """Compiles oracle.c if the library is missing or older than the source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = os.environ.get("CC", "gcc")
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11",
           *_openmp_flag(cc), "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
