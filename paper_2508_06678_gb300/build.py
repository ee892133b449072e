"""Build libqg.so (the CUDA path behind include/qg.h) in-tree for sm_103a.

Each .cu translation unit is compiled in parallel with nvcc, then linked into
``paper_2508_06678_gb300/_build/libqg.so``.  Only the CUDA runtime is linked.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libqg.so")
# the bounds-checked debug build (every shared and global access of the generic row and column passes and their
# FFT is checked; an index outside its array sets a status bit reported as QG_ERR_BOUNDS): tests only
CHECKED_DIR = os.path.join(HERE, "_build_checked")
CHECKED_FLAGS = ("-DQG_CHECKED",)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libqg")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def build(verbose: bool = False, extra_flags=(), out_dir: str = OUT_DIR) -> str:
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    srcs = sources()
    objs = [os.path.join(out_dir, os.path.basename(s)[:-3] + ".o") for s in srcs]

    def compile_one(pair):
        src, obj = pair
        cmd = [cc, *ARCH, *FLAGS, *extra_flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(16, len(srcs), os.cpu_count() or 8)) as ex:
        for msg in ex.map(compile_one, zip(srcs, objs)):
            if verbose and msg:
                print(msg, file=sys.stderr)
    lib = os.path.join(out_dir, "libqg.so")
    tmp = lib + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build_checked(verbose: bool = False) -> str:
    return build(verbose, CHECKED_FLAGS, CHECKED_DIR)


if __name__ == "__main__":
    if "--checked" in sys.argv:
        print(build_checked(verbose="-v" in sys.argv))
    else:
        print(build(verbose="-v" in sys.argv))
