"""Build libwx.so in-tree with nvcc for sm_103a (GB300).

Each translation unit under csrc/ is compiled in parallel, then linked into
``paper_1802_05839_gb300/libwx.so`` (CUDA runtime linked statically, driver
entry points resolved at run time).  No cmake, no torch extension machinery.

``build(bounds=True)`` makes the bounds-checked debug library
``libwx_bounds.so`` from the same sources compiled with ``-DWX_BOUNDS_CHECK``:
every guarded device access checks its element offset against its buffer,
skips it when outside and reports it through the context's status word.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
OBJ_BOUNDS = os.path.join(HERE, "_build_bounds")
LIB = os.path.join(HERE, "libwx.so")
LIB_BOUNDS = os.path.join(HERE, "libwx_bounds.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I" + os.path.join(os.path.dirname(HERE), "include")]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _compile(src: str, extra, obj_dir: str, defines) -> str:
    obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
    if os.path.exists(obj) and not extra:
        deps = [src] + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(
            os.path.join(os.path.dirname(HERE), "include", "*.h"))
        if all(os.path.getmtime(obj) >= os.path.getmtime(d) for d in deps):
            return obj
    cmd = [nvcc(), *ARCH, *FLAGS, *defines, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj


def _link(objs, lib: str, force: bool) -> None:
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < newest:
        r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", lib, *objs], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stderr)


def build(verbose: bool = False, extra=(), bounds: bool = False, both: bool = False) -> str:
    """Build libwx.so (or, with bounds, libwx_bounds.so; with both, the two
    from one parallel compile).  Returns the (first) library's path."""
    variants = [False, True] if both else [bounds]
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    jobs = []
    for b in variants:
        d = OBJ_BOUNDS if b else OBJ
        os.makedirs(d, exist_ok=True)
        jobs += [(s, d, ["-DWX_BOUNDS_CHECK"] if b else []) for s in srcs]
    # the two largest translation units first, so that they overlap the rest
    jobs.sort(key=lambda j: -os.path.getsize(j[0]))
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 8, len(jobs))) as ex:
        objs = list(ex.map(lambda j: (j[1], _compile(j[0], list(extra), j[1], j[2])), jobs))
    for b in variants:
        d = OBJ_BOUNDS if b else OBJ
        lib = LIB_BOUNDS if b else LIB
        _link([o for dd, o in objs if dd == d], lib, bool(extra))
        if verbose:
            print("built", lib)
    return LIB_BOUNDS if (bounds and not both) else LIB


def ptxas_report(src_name: str) -> str:
    """Register / shared-memory report of one translation unit (-Xptxas -v)."""
    src = os.path.join(CSRC, src_name)
    cmd = [nvcc(), *ARCH, *FLAGS, "-Xptxas", "-v", "-c", src, "-o", os.devnull]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return r.stderr


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "ptxas":
        print(ptxas_report(sys.argv[2]))
    elif len(sys.argv) > 1 and sys.argv[1] == "bounds":
        build(verbose=True, bounds=True)
    else:
        build(verbose=True)
