"""Build of the CUDA library: nvcc for sm_103a, one object per translation
unit, compiled in parallel, linked into _build/libspinsum.so (in-tree).
SPINSUM_NVCC_FLAGS adds nvcc flags (e.g. -D overrides of the kernel shape
constants in csrc/ss_internal.h); its -D definitions reach the host sources
too, which size the grids from the same constants."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libspinsum.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _cuda_include() -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(_nvcc()))), "include")


def _commands():
    nvcc = _nvcc()
    cmds = []
    deps = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + [
        os.path.join(INCLUDE, "spinsum.h")]
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
               "-I", INCLUDE, *os.environ.get("SPINSUM_NVCC_FLAGS", "").split(), "-c", src, "-o", obj]
        cmds.append((src, obj, cmd, deps))
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cpp"))):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        defs = [f for f in os.environ.get("SPINSUM_NVCC_FLAGS", "").split() if f.startswith("-D")]
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I", INCLUDE, "-I", _cuda_include(), *defs, "-c",
               src, "-o", obj]
        cmds.append((src, obj, cmd, deps))
    return cmds


def _stale(src, obj, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src, *deps])


def build(verbose: bool = False, force: bool = False, jobs: int | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    # objects built with other SPINSUM_NVCC_FLAGS are stale too
    stamp = os.path.join(BUILD, "flags.txt")
    flags = os.environ.get("SPINSUM_NVCC_FLAGS", "").strip()
    try:
        old = open(stamp).read()
    except OSError:
        old = None
    if old != flags:
        force = True
    todo = [c for c in _commands() if force or _stale(c[0], c[1], c[3])]
    if verbose:
        print(f"[spinsum build] {len(todo)} translation unit(s) to compile")

    def run(c):
        src, obj, cmd, _ = c
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return src

    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            for src in ex.map(run, todo):
                if verbose:
                    print(f"[spinsum build] compiled {os.path.basename(src)}")
    with open(stamp, "w") as f:
        f.write(flags)
    objs = [c[1] for c in _commands()]
    if todo or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        cmd = [_nvcc(), *ARCH, "-shared", "-o", LIB, *objs, "-lrt", "-ldl", "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv)
