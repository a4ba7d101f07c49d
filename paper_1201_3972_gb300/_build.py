"""Build the CUDA library (libirfnr.so) in-tree with nvcc for sm_103a.

Each .cu under csrc/ is compiled to an object in parallel, then the objects
are linked into ``paper_1201_3972_gb300/libirfnr.so``. Objects are rebuilt
when their source or any header is newer.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(ROOT, "_build")
LIB_PATH = os.path.join(PKG, "libirfnr.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
                     "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libirfnr.so")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, obj: str, extra) -> None:
    cmd = [nvcc()] + NVCC_FLAGS + list(extra) + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)


DEBUG_LIB_PATH = os.path.join(PKG, "libirfnr_debug.so")


def build_debug(force: bool = False, verbose: bool = False) -> str:
    """The same library with FNR_DEBUG_CHECKS: kernels check their list
    indices, TMA coordinates and launch layout, record a failure in the status
    word (IR_ECHECK) and skip the access. Built apart, as libirfnr_debug.so;
    load it with IRFNR_LIBRARY=<path>. Returns its path."""
    return build(force, verbose, extra_flags=("-DFNR_DEBUG_CHECKS",), out=DEBUG_LIB_PATH,
                 build_dir=os.path.join(BUILD_DIR, "debug"))


def build(force: bool = False, verbose: bool = False, extra_flags=(), out: str = LIB_PATH,
          build_dir: str = BUILD_DIR) -> str:
    """Compile and link libirfnr.so (or `out`); returns its path."""
    os.makedirs(build_dir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdrs = _headers()
    jobs = []
    objs = []
    for s in srcs:
        o = os.path.join(build_dir, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            jobs.append((s, o))
    if jobs:
        workers = min(len(jobs), max(1, os.cpu_count() or 1))
        with cf.ThreadPoolExecutor(workers) as ex:
            futs = [ex.submit(_compile, s, o, extra_flags) for s, o in jobs]
            for f in futs:
                f.result()
    if force or jobs or _stale(out, objs):
        tmp = out + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, out)
    if verbose:
        print(f"built {out}", file=sys.stderr)
    return out


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
