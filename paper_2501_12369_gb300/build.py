"""Build libdarb.so in-tree with nvcc for sm_103a (GB300).

Each .cu file compiles to an object in parallel, then nvcc links the shared library.
Objects are rebuilt only when a source or header is newer.  No cmake, no torch extension
machinery: the library is a plain C-ABI shared object loaded with ctypes.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(OUT_DIR, "libdarb.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-warn-spills",
                     "--expt-relaxed-constexpr", "-I", CSRC, "-I", INCLUDE]
# Tuning macros (for example -DDARB_SORT_THREADS=256 -DDARB_SORT_CTAS_PER_SM=4), from the
# environment; a change of them rebuilds every object.
DEFINES = os.environ.get("DARB_NVCC_DEFINES", "").split()


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: libdarb.so cannot be built")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return (glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
            glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(target, deps, stamp):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps + [stamp])


def _compile(src, out_dir, defines, stamp, verbose):
    obj = os.path.join(out_dir, os.path.basename(src) + ".o")
    if not _stale(obj, [src] + _headers(), stamp):
        return obj
    cmd = [nvcc()] + NVCC_FLAGS + defines + (["-Xptxas", "-v"] if verbose else []) + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def _build_into(out_dir, lib_path, defines, force, verbose):
    os.makedirs(out_dir, exist_ok=True)
    stamp = os.path.join(out_dir, "defines.txt")
    old = open(stamp).read() if os.path.exists(stamp) else None
    if old != " ".join(defines):
        with open(stamp, "w") as f:
            f.write(" ".join(defines))
    srcs = sources()
    if force:
        for o in glob.glob(os.path.join(out_dir, "*.o")):
            os.remove(o)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(lambda s: _compile(s, out_dir, defines, stamp, verbose), srcs))
    if force or _stale(lib_path, objs, stamp):
        cmd = [nvcc()] + ARCH + ["-shared", "-Xcompiler", "-pthread", "-o", lib_path + ".tmp"] + objs + ["-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc link failed:\n" + r.stderr)
        os.replace(lib_path + ".tmp", lib_path)
    return lib_path


def build(force: bool = False, verbose: bool = False) -> str:
    """libdarb.so, the library every caller loads."""
    return _build_into(OUT_DIR, LIB_PATH, DEFINES, force, verbose)


def build_variant(name: str, defines, force: bool = False) -> str:
    """A separately built copy of the library (its own folder under _build/) with extra macros,
    for tests of build-time paths such as the bounded look-back's timeout."""
    out_dir = os.path.join(OUT_DIR, name)
    return _build_into(out_dir, os.path.join(out_dir, "libdarb.so"), DEFINES + list(defines), force, False)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
