"""In-tree build of libnullspace.so for GB300 (sm_103a) with nvcc.

Each CUDA translation unit is compiled in parallel to an object file, then the
objects are linked into one shared library.  Outputs live under
_build/<machine>/ next to this file, so builds for different host
architectures never mix.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["k_sparse.cu", "k_dense.cu", "k_eig.cu", "k_batched.cu", "ns_api.cu", "ns_batch.cu", "ns_noalloc.cu", "k_peak.cu", "k_umma.cu", "k_dfproj.cu", "k_precond.cu"]
HEADERS = ["ns_common.cuh", "ns_kernels.cuh", "ns_batch.cuh", "ns_checkpoint.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-diag-suppress", "177"]


def build_dir() -> str:
    return os.path.join(HERE, "_build", platform.machine())


def lib_path() -> str:
    return os.path.join(build_dir(), "libnullspace.so")


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnullspace")


def _mtime(p: str) -> float:
    return os.path.getmtime(p) if os.path.exists(p) else -1.0


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if needed) and return the path of libnullspace.so."""
    out_dir = build_dir()
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    deps = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "nullspace.h")]
    dep_time = max(_mtime(p) for p in deps)
    objs, jobs = [], []
    for src in SOURCES:
        sp = os.path.join(CSRC, src)
        op = os.path.join(out_dir, src.replace(".cu", ".o"))
        objs.append(op)
        if force or _mtime(op) < max(_mtime(sp), dep_time):
            jobs.append([nvcc, *ARCH, *FLAGS, "-c", sp, "-o", op])
    lib = lib_path()

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(run, jobs))
    if jobs or _mtime(lib) < max(_mtime(o) for o in objs):
        tmp = lib + ".tmp"
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
