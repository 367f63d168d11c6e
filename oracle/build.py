"""Build the WASABI oracle shared library (test infrastructure only).

Compiles ``wasabi_oracle.cpp`` with the host C++ compiler into
``oracle/_build/liboracle.so``.  Floating-point contraction is switched off:
the FP32 selection path depends on every rounding being the one written in
the source.  OpenMP is used when the compiler supports it (it only splits
independent depths / output rows across threads and never changes a result).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "wasabi_oracle.cpp")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def _compile(extra: list[str], out: str) -> subprocess.CompletedProcess:
    cxx = os.environ.get("CXX", shutil.which("g++") or "c++")
    cmd = [cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", *extra, SRC, "-o", out]
    return subprocess.run(cmd, capture_output=True, text=True)


def build(force: bool = False) -> str:
    """Compile the oracle if it is missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    res = _compile(["-fopenmp"], tmp)
    if res.returncode != 0:
        res = _compile([], tmp)
    if res.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + res.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
