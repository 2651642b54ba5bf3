"""Build the in-tree CUDA library liblbmadj.so for sm_103a with nvcc.

    python -m paper_2608_19617_b300.build [--force]

The library is written next to this file so that it travels with the source
tree; it is rebuilt when any source under csrc/ or include/ is newer.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "liblbmadj.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_FILES = ("lbmadj.cu", "noalloc.cu", "mma.cu")


def _sources():
    out = []
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            if name.endswith((".cu", ".cuh", ".h")):
                out.append(os.path.join(d, name))
    return out


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def command(out=LIB, extra=()):
    return [nvcc_path(), "-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-O3",
            "--shared", "-cudart", "shared", "-I", INCLUDE, "-I", CSRC, *extra,
            *[os.path.join(CSRC, f) for f in CU_FILES], "-o", out]


def build(force: bool = False, verbose: bool = False) -> str:
    srcs = _sources()
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return LIB
    cmd = command()
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    tmp = LIB + ".tmp"
    cmd[-1] = tmp
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stdout + res.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
