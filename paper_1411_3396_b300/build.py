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
LIB_CHECKED = PKG / "libsr_b300_check.so"     # bounds-checked build (-DSR_CHECK)
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


def needs_build(lib: Path = LIB) -> bool:
    if not lib.exists():
        return True
    t = lib.stat().st_mtime
    return any(f.stat().st_mtime > t for f in _inputs())


def _compile(targets, verbose, extra):
    """Compile every source of each (library, extra flags) target to objects
    (all in parallel), then link each library."""
    with tempfile.TemporaryDirectory(prefix="sr_build_") as d:
        jobs, links = [], []
        for k, (lib, flags_extra) in enumerate(targets):
            flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", str(INCLUDE),
                     *flags_extra, *(extra or [])]
            objs = [os.path.join(d, f"{k}_{s}.o") for s in SOURCES]
            jobs += [[_nvcc(), *flags, "-c", str(CSRC / s), "-o", o] for s, o in zip(SOURCES, objs)]
            links.append((lib, [_nvcc(), *ARCH, "-shared", "-o", str(lib.with_suffix(".so.tmp")), *objs]))
        with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, res in zip(jobs, results):
            if verbose or res.returncode != 0:
                print(" ".join(cmd))
                print(res.stdout)
                print(res.stderr)
            if res.returncode != 0:
                raise RuntimeError("nvcc failed building the library:\n" + res.stderr[-4000:])
        for lib, cmd in links:
            res = subprocess.run(cmd, capture_output=True, text=True)
            if verbose or res.returncode != 0:
                print(" ".join(cmd))
                print(res.stdout)
                print(res.stderr)
            if res.returncode != 0:
                raise RuntimeError("nvcc failed linking " + lib.name + ":\n" + res.stderr[-4000:])
            os.replace(lib.with_suffix(".so.tmp"), lib)


def build(force: bool = False, verbose: bool = False, extra=None, checked: bool = True) -> Path:
    """Build libsr_b300.so and (checked=True) the bounds-checked
    libsr_b300_check.so where a source is newer than the library."""
    targets = []
    if force or needs_build(LIB):
        targets.append((LIB, []))
    if checked and (force or needs_build(LIB_CHECKED)):
        targets.append((LIB_CHECKED, ["-DSR_CHECK"]))
    if targets:
        _compile(targets, verbose, extra)
    return LIB


if __name__ == "__main__":
    import sys
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None)
