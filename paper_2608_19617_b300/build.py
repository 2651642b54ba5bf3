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


def _compile_cmd(src, obj, extra=()):
    return [nvcc_path(), "-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-O3",
            "-I", INCLUDE, "-I", CSRC, *extra, "-c", src, "-o", obj]


def command(out=LIB, extra=()):
    """One nvcc invocation that compiles and links every source (for reference;
    build() compiles the files in parallel and links them)."""
    return [nvcc_path(), "-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-O3",
            "--shared", "-cudart", "shared", "-I", INCLUDE, "-I", CSRC, *extra,
            *[os.path.join(CSRC, f) for f in CU_FILES], "-o", out]


def build(force: bool = False, verbose: bool = False) -> str:
    srcs = _sources()
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return LIB
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    procs = []
    for f in CU_FILES:
        obj = os.path.join(objdir, f + ".o")
        cmd = _compile_cmd(os.path.join(CSRC, f), obj)
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)))
    objs = []
    for cmd, obj, p in procs:
        out, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + out + err)
        objs.append(obj)
    tmp = LIB + ".tmp"
    link = [nvcc_path(), *ARCH, "--shared", "-cudart", "shared", *objs, "-o", tmp]
    if verbose:
        print(" ".join(link), file=sys.stderr)
    res = subprocess.run(link, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + res.stdout + res.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
