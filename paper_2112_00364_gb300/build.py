"""Build the CUDA library ``libsmc.so`` in-tree for sm_103a (GB300).

Each .cu file is compiled by nvcc in parallel (one -gencode, -lineinfo,
-fmad=false so that every fused multiply-add in the kernels is an explicit
fma() of the specification) and the objects are linked into one shared
library next to this file.  The checking build ``libsmc_debug.so`` is the same
sources compiled with SMC_DEBUG_CHECKS=1: every ancestor index, gathered block
index and stack pointer is checked, and an out-of-range one is recorded in the
run's counters and skipped instead of accessed.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
INCLUDE = PKG.parent / "include"
BUILD = PKG / "_build"
LIB = PKG / "libsmc.so"
LIB_DEBUG = PKG / "libsmc_debug.so"
SOURCES = ["smc_engine.cu", "smc_waves_kind.cu", "smc_small.cu", "smc_prims.cu", "smc_server.cu",
           "smc_probe.cu"]
GENCODE = "arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsmc.so")


def _flags() -> list[str]:
    return ["-gencode", GENCODE, "-O3", "-lineinfo", "-std=c++17", "-fmad=false",
            "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-I", str(INCLUDE), "-I", str(CSRC)]


def _deps() -> list[Path]:
    return sorted(CSRC.glob("*.cu")) + sorted(CSRC.glob("*.cuh")) + sorted(CSRC.glob("*.h")) + \
        sorted(INCLUDE.glob("*.h")) + [Path(__file__)]


def up_to_date(lib: Path = LIB) -> bool:
    if not lib.exists():
        return False
    t = lib.stat().st_mtime
    return all(p.stat().st_mtime <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False,
          debug: bool = False) -> Path:
    """Build libsmc.so (debug=True: the checking build libsmc_debug.so)."""
    lib = LIB_DEBUG if debug else LIB
    if not force and up_to_date(lib):
        return lib
    out = BUILD / ("debug" if debug else "release")
    out.mkdir(parents=True, exist_ok=True)
    cc = nvcc()
    extra = (["-Xptxas", "-v"] if ptxas_v else []) + (["-DSMC_DEBUG_CHECKS=1"] if debug else [])

    def compile_one(src: str):
        obj = out / (Path(src).stem + ".o")
        cmd = [cc, "-c", str(CSRC / src), "-o", str(obj)] + _flags() + extra
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{p.stderr}")
        return obj, p.stderr

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_v:
        for _, err in results:
            if err:
                print(err)
    tmp = lib.with_suffix(f".so.tmp{os.getpid()}")
    cmd = [cc, "-shared", "-o", str(tmp)] + [str(o) for o, _ in results] + \
        ["-gencode", GENCODE, "-Xcompiler", "-fPIC", "-lcudart"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stderr}")
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> list[Path]:
    """Both libraries, compiled at the same time."""
    with ThreadPoolExecutor(max_workers=2) as ex:
        return list(ex.map(lambda d: build(force=force, debug=d), (False, True)))


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv,
                debug="--debug" in sys.argv))
