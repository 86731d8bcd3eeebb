"""Builds the CUDA library liblbm.so for sm_103a (GB300) in-tree.

nvcc compiles the translation units in parallel and links them with
the static CUDA runtime; the result lands in paper_2101_01702_gb300/_build.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = BUILD / "liblbm.so"
LIB_CHECKED = BUILD / "liblbm_checked.so"   # every geometry-derived index checked (tests)
SOURCES = ["lbm_api.cu", "k_fp64.cu", "k_mixed.cu", "k_mixed_fast.cu", "k_fixed_scratch.cu", "k_probe.cu", "k_adjoint.cu",
           "k_persist_fp64.cu", "k_persist_mixed.cu", "k_persist_mixed_fast.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = Path(cuda) / "bin" / "nvcc"
    return str(cand) if cand.exists() else "nvcc"


def _inputs():
    return [CSRC / s for s in SOURCES] + sorted(CSRC.glob("*.cuh")) + sorted(CSRC.glob("*.h")) + [
        PKG.parent / "include" / "lbm.h"]


def up_to_date(lib: Path = LIB) -> bool:
    if not lib.exists():
        return False
    t = lib.stat().st_mtime
    return all(p.stat().st_mtime <= t for p in _inputs())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> Path:
    """Builds liblbm.so, or with checked=True liblbm_checked.so: the same
    library compiled with LBMK_CHECKED=1, whose kernels check every index
    they derive from the lattice geometry and report LBM_ERR_BOUNDS."""
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(lib):
        return lib
    BUILD.mkdir(exist_ok=True)
    nvcc = _nvcc()
    tag = os.getpid()

    def compile_one(src: str):
        obj = BUILD / f"{Path(src).stem}.{tag}{'.checked' if checked else ''}.o"
        cmd = [nvcc, *ARCH, *FLAGS, *(["-DLBMK_CHECKED=1"] if checked else []), "-I", str(PKG.parent / "include"),
               "-c", str(CSRC / src), "-o", str(obj)]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = BUILD / f"{lib.stem}.{tag}.so"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", str(tmp), *map(str, objs)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    for o in objs:
        o.unlink(missing_ok=True)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
