"""Build libllb.so in-tree with nvcc for sm_103a.

Each translation unit under ``csrc/`` is compiled in parallel into
``_build/`` and linked into ``libllb.so`` next to this file.  No cmake, no
torch extension machinery: the library is a plain C-ABI shared object.

``build(checked=True)`` compiles the same sources with ``-DLLB_CHECKED`` into
``_build_checked/`` and ``libllb_checked.so``: every stencil-kernel index is
compared with its buffer's extent and an out-of-range access is skipped and
recorded (``llb_checked_status``) instead of touching memory.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libllb.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libllb_checked.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fvisibility=hidden"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libllb")
    return path


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(INCLUDE, "llb.h"))
    return hs


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra, bdir: str) -> str:
    obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
    if _stale(obj, [src] + _headers()):
        cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
    return obj


def build(verbose: bool = False, extra=None, force: bool = False, checked: bool = False,
          pool: cf.Executor | None = None) -> str:
    """Compile and link libllb.so (libllb_checked.so if checked); returns its
    path.  Incremental unless force."""
    extra = list(extra or [])
    bdir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    if checked:
        extra.append("-DLLB_CHECKED")
    os.makedirs(bdir, exist_ok=True)
    if force:
        for f in os.listdir(bdir):
            os.remove(os.path.join(bdir, f))
    srcs = sources()
    own = pool is None
    ex = pool or cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4))
    try:
        objs = list(ex.map(lambda s: _compile(s, extra, bdir), srcs))
    finally:
        if own:
            ex.shutdown()
    if force or _stale(lib, objs):
        tmp = lib + ".tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}", file=sys.stderr)
    return lib


def build_all(verbose: bool = False, force: bool = False):
    """Both libraries, their translation units compiled by one pool."""
    n = 2 * len(sources())
    with cf.ThreadPoolExecutor(max_workers=min(n, os.cpu_count() or 4)) as pool, \
            cf.ThreadPoolExecutor(max_workers=2) as outer:
        futs = [outer.submit(build, verbose, None, force, chk, pool) for chk in (False, True)]
        return [f.result() for f in futs]


if __name__ == "__main__":
    if "--checked" in sys.argv:
        build(verbose=True, force="--force" in sys.argv, checked=True)
    else:
        build(verbose=True, force="--force" in sys.argv)
