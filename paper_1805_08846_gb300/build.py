"""Build the CUDA library libclaw.so in-tree for sm_103a (GB300).

Each translation unit under csrc/ is compiled by nvcc in parallel
(``-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo``) and linked
into ``paper_1805_08846_gb300/_build/libclaw.so``.  ``build(debug=True)``
makes the checked variant (``-DCLAW_DEBUG``: bounds checks of every direct
global access and bulk-copy coordinate in the kernels) in
``_build_debug/libclaw.so``.  Nothing is installed outside this directory.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libclaw.so")
OUT_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(OUT_DEBUG, "libclaw.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hs + [os.path.join(INCLUDE, "claw.h"), os.path.abspath(__file__)]


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in sources()] + headers()
    return any(os.path.getmtime(p) > t for p in deps)


def flags():
    return [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
            "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _compile(src: str, verbose: bool, extra, out: str = OUT) -> str:
    obj = os.path.join(out, src[:-3] + ".o")
    cmd = [nvcc()] + flags() + list(extra) + ["-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    if verbose and r.stderr:
        print(r.stderr, file=sys.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, extra=(), debug: bool = False) -> str:
    out, lib = (OUT_DEBUG, LIB_DEBUG) if debug else (OUT, LIB)
    if debug:
        extra = list(extra) + ["-DCLAW_DEBUG"]
    if not force and not _stale(lib):
        return lib
    os.makedirs(out, exist_ok=True)
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, extra, out), srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), ARCH, "-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=True, verbose=v, extra=extra))
