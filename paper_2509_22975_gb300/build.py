"""Build libmcd.so (the C-ABI library) for sm_103a, in-tree.

Each translation unit is compiled by nvcc in its own process (in parallel),
then linked into paper_2509_22975_gb300/_build/libmcd.so.  The CUDA runtime is
linked statically, so the library only needs the driver at run time.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libmcd.so")
SOURCES = ["mcd_api.cu", "index.cu", "hv.cu", "hv_hash.cu", "hv_cache.cu", "hv_cache_cols.cu", "hv_cache_items.cu", "krylov.cu", "band.cu", "adjoint.cu", "noalloc.cu", "sampler.cpp", "sampler_gpu.cu", "batch.cu", "tridiag.cpp",
           "symeig.cpp", "basis_io.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _flags(src: str) -> list[str]:
    f = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O3,-Wall", "-I" + os.path.join(HERE, "..", "include")]
    if src.endswith(".cu"):
        f += ARCH + ["-lineinfo", "--expt-relaxed-constexpr"]
    return f


def _newer(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(d) <= t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    headers = [os.path.join(SRC, h) for h in os.listdir(SRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(HERE, "..", "include", "mcd.h"))
    objs = []
    jobs = []
    for s in SOURCES:
        src = os.path.join(SRC, s)
        obj = os.path.join(OUT, s + ".o")
        objs.append(obj)
        if force or not _newer(obj, [src] + headers + [__file__]):
            jobs.append([NVCC, "-c", src, "-o", obj] + _flags(s))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {cmd[2]}")
        return r

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    if force or jobs or not _newer(LIB, objs):
        run([NVCC, "-shared", "-o", LIB] + objs + ARCH + ["-Xcompiler", "-fPIC", "-lpthread"])
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
