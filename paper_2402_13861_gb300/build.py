"""Builds the CUDA library ``libisx.so`` for sm_103a in place (no torch extension machinery: the
library exposes a plain C interface).  Translation units compile in parallel."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = PKG / "libisx.so"
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found")


def common_flags(debug=False):
    flags = [ARCH, "-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
             "-Xptxas", "-warn-spills"]
    if debug:
        flags += ["-DISX_DEBUG=1"]
    return flags


def _stamp(paths):
    return max(p.stat().st_mtime for p in paths)


def build(force=False, verbose=False, debug=False):
    srcs = sorted(CSRC.glob("*.cu"))
    headers = sorted(CSRC.glob("*.cuh")) + sorted((PKG.parent / "include").glob("*.h"))
    BUILD.mkdir(exist_ok=True)
    cc = nvcc()
    hdr_time = _stamp(headers)

    def compile_one(src):
        obj = BUILD / (src.stem + ".o")
        if not force and obj.exists() and obj.stat().st_mtime >= max(src.stat().st_mtime, hdr_time):
            return None
        cmd = [cc, *common_flags(debug), "-c", str(src), "-o", str(obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src.name}:\n{r.stdout}\n{r.stderr}")
        return r.stderr if verbose else None

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        logs = list(ex.map(compile_one, srcs))
    if verbose:
        for s, log in zip(srcs, logs):
            if log:
                print(f"--- {s.name}\n{log}")
    objs = [BUILD / (s.stem + ".o") for s in srcs]
    if force or not LIB.exists() or LIB.stat().st_mtime < _stamp(objs):
        cmd = [cc, ARCH, "-shared", "-o", str(LIB), *map(str, objs)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
