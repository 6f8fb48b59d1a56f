"""Build the CUDA C-ABI library for sm_103a (in-tree, no cmake).

Compiles each translation unit of csrc/ with nvcc in parallel and links
paper_2201_06039_gb300/_build/libgb300lbm.so, and the same sources with -DLBM_BOUNDS_CHECK into
paper_2201_06039_gb300/_build/bounds/libgb300lbm_bounds.so (every kernel index checked before use;
for debugging and its GPU test, not for timing).  Rebuilds only when a source changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libgb300lbm.so")
BOUNDS_DIR = os.path.join(OUT_DIR, "bounds")
BOUNDS_LIB = os.path.join(BOUNDS_DIR, "libgb300lbm_bounds.so")
VARIANTS = {"release": (OUT_DIR, LIB, ()), "bounds": (BOUNDS_DIR, BOUNDS_LIB, ("-DLBM_BOUNDS_CHECK",))}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(ROOT, "include", "lbm.h"), os.path.abspath(__file__)]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), variants=("release", "bounds")) -> str:
    """Build the requested library variants (all translation units of all variants compile in
    parallel); returns the path of the release library."""
    todo = [v for v in variants if force or extra_flags or not up_to_date(VARIANTS[v][1])]
    if not todo:
        return LIB
    cc = nvcc()
    jobs = []
    for v in todo:
        out_dir, _, vflags = VARIANTS[v]
        os.makedirs(out_dir, exist_ok=True)
        for src in _sources():
            jobs.append((v, src, os.path.join(out_dir, os.path.basename(src) + ".o"), (*vflags, *extra_flags)))

    def compile_one(job):
        v, src, obj, flags = job
        cmd = [cc, *ARCH, *FLAGS, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)} ({v}):\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        list(ex.map(compile_one, jobs))
    for v in todo:
        out_dir, lib, _ = VARIANTS[v]
        objs = [os.path.join(out_dir, os.path.basename(src) + ".o") for src in _sources()]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed ({v}):\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
