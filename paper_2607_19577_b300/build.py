"""Build libqst.so (the C-ABI library) in-tree for sm_103a with nvcc."""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
SRC = PKG / "csrc" / "qst.cu"
HDR = ROOT / "include" / "qst.h"
LIB = PKG / "libqst.so"
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-shared", "-I", str(ROOT / "include")]


def build(force: bool = False, verbose: bool = False) -> Path:
    deps = [SRC, HDR, *sorted((PKG / "csrc").glob("*.cuh"))]
    stale = not LIB.exists() or LIB.stat().st_mtime < max(d.stat().st_mtime for d in deps)
    if force or stale:
        tmp = LIB.with_suffix(".so.tmp%d" % os.getpid())
        cmd = [NVCC, *FLAGS, *(["-Xptxas", "-v"] if verbose else []), "-o", str(tmp), str(SRC)]
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
