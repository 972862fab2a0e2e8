"""Build the C-ABI library libep.so in-tree for sm_103a (nvcc + g++, no cmake).

Each translation unit is compiled in parallel, then linked with nvcc:
    nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo -Xcompiler -fPIC -shared
The output goes to paper_1805_04155_gb300/_lib/libep.so (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libep.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libep.so")


def sources():
    cu = sorted(f for f in os.listdir(SRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(SRC) if f.endswith(".cpp"))
    return cu, cpp


def _compile(args):
    cmd, src = args
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compiling {src} failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return src


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile every source under csrc/ and link libep.so; returns the library path."""
    cu, cpp = sources()
    os.makedirs(OUT_DIR, exist_ok=True)
    obj_dir = os.path.join(OUT_DIR, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(HERE, "..", "include", "ep.h")]
    newest = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    nvcc = _nvcc()
    common = ["-std=c++17", "-O3", "-Xcompiler", "-fPIC", "-I", os.path.join(HERE, "..", "include")]
    jobs_list = []
    objs = []
    for f in cu:
        o = os.path.join(obj_dir, f[:-3] + ".o")
        objs.append(o)
        jobs_list.append(([nvcc, *ARCH, "-lineinfo", *common, "-c", os.path.join(SRC, f), "-o", o], f))
    for f in cpp:
        o = os.path.join(obj_dir, f[:-4] + ".o")
        objs.append(o)
        jobs_list.append(([nvcc, *common, "-Xcompiler", "-fopenmp", "-x", "c++", "-c", os.path.join(SRC, f), "-o", o], f))
    jobs = jobs or max(2, min(len(jobs_list), os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        for src in ex.map(_compile, jobs_list):
            if verbose:
                print(f"  compiled {src}", file=sys.stderr)
    tmp = LIB + ".tmp"
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-Xcompiler", "-fopenmp"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"linking libep.so failed:\n{' '.join(link)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
