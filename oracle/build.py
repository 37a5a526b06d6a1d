"""Compile the CPU oracle into oracle/_build/liborc.so with gcc.

Test infrastructure only.  Flags: -O2 -ffp-contract=off (no fused
multiply-add, on x86-64 or aarch64 alike), OpenMP over independent lines.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["orc_acoustics.c", "orc_shallow_water.c", "orc_wavesweep.c", "orc_unsplit.c"]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liborc.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["orc.h", "build.py"]
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = os.environ.get("CC", "gcc")
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-fopenmp", "-shared", "-Wall", "-o", tmp]
    cmd += [os.path.join(HERE, s) for s in SOURCES] + ["-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
