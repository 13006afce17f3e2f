"""Builds the C-ABI shared library librecon.so for sm_103a (nvcc, in-tree)."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "librecon.so")
SOURCES = ["recon_kernels.cu", "recon_api.cu", "recon_sched.cu", "recon_learn.cu", "recon_noalloc.cu",
           "recon_mb.cu", "recon_dt.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _deps() -> list:
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hdrs + [os.path.join(ROOT, "include", "recon.h")]


LIB_CHECKS = os.path.join(PKG, "librecon_checks.so")


def build(force: bool = False, verbose: bool = False, checks: bool = False) -> str:
    """Builds librecon.so; checks=True builds the bounds-checked variant
    librecon_checks.so instead (-DRECON_CHECKS, see recon_checks in recon.h)."""
    bdir = BUILD + ("_checks" if checks else "")
    lib_path = LIB_CHECKS if checks else LIB
    extra = ["-DRECON_CHECKS"] if checks else []
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    dep_mtime = max(os.path.getmtime(p) for p in _deps())

    def compile_one(src: str) -> str:
        s = os.path.join(CSRC, src)
        o = os.path.join(bdir, src.replace(".cu", ".o"))
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), dep_mtime):
            cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", s, "-o", o + ".tmp"]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            subprocess.check_call(cmd)
            os.replace(o + ".tmp", o)
        return o

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    if force or not os.path.exists(lib_path) or os.path.getmtime(lib_path) < max(os.path.getmtime(o) for o in objs):
        tmp = lib_path + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs])
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
