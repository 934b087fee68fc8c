"""Compile libsfg.so in-tree for sm_103a (GB300) with nvcc.

build.cu (frame, keys, sort, octree, FP64 moments) is compiled without FMA
contraction so that its FP64 results are reproducible operation by operation;
the walk/eval file may contract FP32 multiply-adds, and its FP32 arithmetic
flushes denormals and uses the hardware reciprocal square root and
approximate division (the FP32 pair terms never come near the denormal
range: positions are offsets of at most 2^22 half-cells and separations of
coincident points are handled before any division).

Environment: SFG_NVCC_EXTRA adds nvcc flags (e.g. -D defines) and
SFG_LIB_NAME names the output library (default libsfg.so), so that builds
with different flags can sit side by side in _lib/.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, os.environ.get("SFG_LIB_NAME", "libsfg.so"))
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-strict-aliasing",
          "--expt-relaxed-constexpr", "-I", INCLUDE]
SOURCES = {
    "build.cu": ["-fmad=false"],
    "walk.cu": ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"],
    "api.cu": [],
}


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsfg")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "sfg.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    os.makedirs(LIBDIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    nvcc = _nvcc()
    extra = list(extra_flags or []) + os.environ.get("SFG_NVCC_EXTRA", "").split()

    def compile_one(name: str) -> str:
        src = os.path.join(CSRC, name)
        stem = os.path.splitext(os.path.basename(LIB))[0]
        obj = os.path.join(LIBDIR, f"{stem}.{name.replace('.cu', '.o')}")
        cmd = [nvcc, "-c", src, "-o", obj] + ARCH + COMMON + SOURCES[name] + extra
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{res.stderr}")
        if verbose:
            print(res.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True, extra_flags=["-Xptxas", "-v"]))
