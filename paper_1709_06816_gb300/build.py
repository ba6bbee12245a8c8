"""Build liblw.so in-tree with nvcc for sm_103a (GB300).

    python -m paper_1709_06816_gb300.build        # or __graft_entry__.build()

Each CUDA translation unit is compiled in parallel (nvcc -c), then linked
into ``paper_1709_06816_gb300/liblw.so``.  Flags: one -gencode for
compute_103a/sm_103a, -O3, -lineinfo, and -fmad=false so that no product and
sum of the update formula is contracted into a fused multiply-add (the
kernels also spell every rounding out with __fmul_rn / __fadd_rn).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(HERE, "liblw.so")
# the bounds-checked variant (-DLW_CHECKED: every global access of the merge
# kernel checked against the job's buffers), built on request for testing
CHECKED_LIB_PATH = os.path.join(HERE, "liblw_checked.so")
SOURCES = ["lw_merge.cu", "lw_api.cu", "lw_noalloc.cu", "lw_server.cu"]
HEADERS = ["lw_internal.h", os.path.join("..", "..", "include", "lw.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-Wall", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblw.so")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, checked: bool = False) -> str:
    """Compile every translation unit (in parallel) and link liblw.so, or,
    with checked=True, liblw_checked.so built with -DLW_CHECKED."""
    nvcc = _nvcc()
    build_dir = os.path.join(BUILD_DIR, "checked") if checked else BUILD_DIR
    lib_path = CHECKED_LIB_PATH if checked else LIB_PATH
    extra = ["-DLW_CHECKED"] if checked else []
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in HEADERS]
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or ptxas_info or _stale(o, [s] + headers):
            cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", s, "-o", o]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_info:
            sys.stdout.write(r.stdout + r.stderr)

    with ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        list(ex.map(run, jobs))
    if jobs or force or _stale(lib_path, objs):
        tmp = lib_path + f".tmp{os.getpid()}"
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                checked="--checked" in sys.argv))
