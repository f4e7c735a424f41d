"""Build the in-tree CUDA library ``_lib/libpg.so`` for sm_103a with nvcc.

The translation units compile in parallel, then link into one shared library
that uses the shared CUDA runtime (so a process that already loaded PyTorch's
``libcudart.so.13`` shares that instance, its context and current device).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libpg.so")
SOURCES = ["pg_kernels.cu", "pg_api.cpp", "pg_build.cpp", "pg_noalloc.cu", "pg_tune.cpp", "pg_init.cpp",
           "pg_domain.cu", "pg_scenarios.cu"]
HEADERS = [os.path.join(CSRC, "pg_internal.h"), os.path.join(CSRC, "pg_grid.h"), os.path.join(CSRC, "pg_device.cuh"),
           os.path.join(ROOT, "include", "pg.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(LIBDIR, exist_ok=True)
    objs, procs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(LIBDIR, src + ".o")
        objs.append(o)
        if force or _stale(o, [s] + HEADERS):
            cmd = [NVCC, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                   "-cudart", "shared", *os.environ.get("PG_EXTRA_NVCC_FLAGS", "").split(), "-c", s, "-o", o]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed ({' '.join(cmd)}):\n{out.decode(errors='replace')}")
        if verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if force or procs or _stale(LIB, objs):
        cmd = [NVCC, *ARCH, "-shared", "-cudart", "shared", *objs, "-o", LIB,
               "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout.decode(errors='replace')}")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
