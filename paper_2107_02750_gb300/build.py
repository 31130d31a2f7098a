"""In-tree build of the CUDA library libmwdg (sm_103a) with nvcc.

The translation units compile in parallel; the FP64 kernels (the solver's
and the adjoint's) are built without FMA contraction (-fmad=false) so that their arithmetic rounds as
written, the FP32 kernels with fast division and square root.  Output: paper_2107_02750_gb300/_build/libmwdg_<machine>.so.
"""
from __future__ import annotations

import os
import platform
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
INCLUDE = ROOT / "include"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = {
    "mwdg_api.cu": [],
    "mwdg_f64.cu": ["-fmad=false"],
    "mwdg_f32.cu": ["--use_fast_math"],
    "mwdg_noalloc.cu": [],
    "mwdg_peaks.cu": [],
    "mwdg_adjoint.cu": ["-fmad=false"],
}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (Path(c).exists() or c == "nvcc"):
            return c
    return "nvcc"


def lib_path() -> Path:
    return BUILD / f"libmwdg_{platform.machine()}.so"


def _sources():
    return sorted(CSRC.glob("*.cu")) + sorted(CSRC.glob("*.cuh")) + sorted(CSRC.glob("*.h")) + sorted(INCLUDE.glob("*.h"))


def up_to_date() -> bool:
    out = lib_path()
    if not out.exists():
        return False
    t = out.stat().st_mtime
    return all(s.stat().st_mtime <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> Path:
    out = lib_path()
    if not force and up_to_date():
        return out
    BUILD.mkdir(exist_ok=True)
    common = ["-std=c++17", "-O3", "-lineinfo", *ARCH, f"-I{INCLUDE}", f"-I{CSRC}",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"]
    objs = []

    def compile_unit(item):
        name, extra = item
        obj = BUILD / (Path(name).stem + f"_{platform.machine()}.o")
        cmd = [nvcc(), *common, *extra, "-c", str(CSRC / name), "-o", str(obj)]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS.items()))
    tmp = out.with_suffix(f".{os.getpid()}.tmp")
    cmd = [nvcc(), *ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
