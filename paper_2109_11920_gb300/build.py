"""Build the in-tree CUDA library ``libboac.so`` for GB300 (sm_103a).

Each ``csrc/*.cu`` is compiled to an object in parallel with nvcc, then the
objects are linked into ``paper_2109_11920_gb300/libboac.so``.  No CMake, no
torch extension machinery: the library is a plain C ABI (``include/boac.h``).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libboac.so")
CHECKED_LIB = os.path.join(PKG, "libboac_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the BOAC CUDA library cannot be built")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hs + [os.path.join(ROOT, "include", "boac.h")]


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra, build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
    if _stale(obj, [src] + headers() + [__file__]):
        cmd = [nvcc()] + ARCH + NVCC_FLAGS + list(extra) + ["-c", src, "-o", obj]
        subprocess.check_call(cmd)
    return obj


def build(force: bool = False, extra_flags=(), verbose: bool = False, checked: bool = False) -> str:
    """Compile and link libboac.so if any source changed; returns its path.
    checked=True builds libboac_checked.so instead: the same library with
    -DBOAC_CHECKED (index checks in the gathers and scatters that count a
    fault and skip the access; boac_bounds_faults reads the count)."""
    build_dir = BUILD + "_checked" if checked else BUILD
    lib = CHECKED_LIB if checked else LIB
    extra_flags = tuple(extra_flags) + (("-DBOAC_CHECKED",) if checked else ())
    os.makedirs(build_dir, exist_ok=True)
    srcs = sources()
    if force:
        for f in os.listdir(build_dir):
            if f.endswith(".o"):
                os.remove(os.path.join(build_dir, f))
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra_flags, build_dir), srcs))
    LIB_OUT = lib
    if force or _stale(LIB_OUT, objs):
        tmp = LIB_OUT + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-ldl"])
        os.replace(tmp, LIB_OUT)
    if verbose:
        print("built", LIB_OUT, file=sys.stderr)
    return LIB_OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv)
