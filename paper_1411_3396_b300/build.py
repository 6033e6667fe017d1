"""Build the native library (CUDA for sm_103a plus host C++) in-tree.

The shared object ``libsr_b300.so`` is written next to this file; the
Python binding loads it from there.  ``build()`` recompiles only when a
source or the public header is newer than the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
LIB = PKG / "libsr_b300.so"
SOURCES = ["abi.cu", "fit.cpp", "radix.cu", "bin.cu", "force.cu", "force_grp.cu", "plain.cu", "kick.cu", "noalloc.cu",
           "centers.cu", "pm.cu", "fof.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsr_b300.so")


def _inputs():
    files = [CSRC / s for s in SOURCES] + list(CSRC.glob("*.h")) + list(CSRC.glob("*.cuh")) + list(INCLUDE.glob("*.h"))
    return files


def needs_build() -> bool:
    if not LIB.exists():
        return True
    t = LIB.stat().st_mtime
    return any(f.stat().st_mtime > t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra=None) -> Path:
    """Compile every source to an object (in parallel), then link."""
    if not force and not needs_build():
        return LIB
    tmp = LIB.with_suffix(".so.tmp")
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", str(INCLUDE), *(extra or [])]
    with tempfile.TemporaryDirectory(prefix="sr_build_") as d:
        objs = [os.path.join(d, s + ".o") for s in SOURCES]
        cmds = [[_nvcc(), *flags, "-c", str(CSRC / s), "-o", o] for s, o in zip(SOURCES, objs)]
        with ThreadPoolExecutor(max_workers=max(1, min(len(cmds), os.cpu_count() or 1))) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), cmds))
        link = [_nvcc(), *ARCH, "-shared", "-o", str(tmp), *objs]
        results.append(subprocess.run(link, capture_output=True, text=True))
        for cmd, res in zip(cmds + [link], results):
            if verbose or res.returncode != 0:
                print(" ".join(cmd))
                print(res.stdout)
                print(res.stderr)
            if res.returncode != 0:
                raise RuntimeError("nvcc failed building libsr_b300.so:\n" + res.stderr[-4000:])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None)
