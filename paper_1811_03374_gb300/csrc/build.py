"""Builds libfiberx.so (sm_103a CUDA kernels + host C ABI) in-tree with nvcc.

Translation units compile in parallel; the result is linked with the static
CUDA runtime.  Used by ``__graft_entry__.build()`` and, when the library is
missing or stale, by the binding on first load.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
PKG = os.path.dirname(HERE)
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "libfiberx.so")
SOURCES = ["filter_kernels.cu", "lane_kernels.cu", "scan_kernels.cu", "ray_kernels.cu", "normal_kernels.cu", "count_kernels.cu", "trace_kernels.cu", "warp_kernels.cu", "backward.cu", "fiberx_api.cu",
           "noalloc.cu", "peak.cu", "presplit.cpp"]
HEADERS = ["trace.cuh", "internal.h", "presplit.h", os.path.join(ROOT, "include", "fiberx.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(HERE, s) for s in SOURCES + HEADERS[:-1]] + [HEADERS[-1]]
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra: list[str] | None = None, out: str | None = None,
          obj_dir: str | None = None) -> str:
    """Compiles and links the library; `extra` nvcc flags, `out` / `obj_dir`
    redirect the result (default: the in-tree libfiberx.so)."""
    lib = out or LIB
    out_dir = obj_dir or os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                     "-I", os.path.join(ROOT, "include")] + (extra or [])

    def one(src):
        obj = os.path.join(out_dir, src + ".o")
        cmd = [cc] + common + ["-c", os.path.join(HERE, src), "-o", obj]
        if verbose and src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(one, SOURCES))
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    if verbose:
        for _, log in results:
            if log:
                print(log)
    return lib


if __name__ == "__main__":
    import sys
    build(verbose="-v" in sys.argv)
    print(LIB)
