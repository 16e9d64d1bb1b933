"""Build the CUDA library ``liblbmp.so`` in-tree for sm_103a (GB300).

The translation units are compiled in parallel with nvcc and linked into a
shared library with the CUDA runtime linked statically, so the library only
needs the NVIDIA driver at run time.  No torch headers are involved: the
library exposes a plain C ABI (``include/lbmp.h``).
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "liblbmp.so")
SOURCES = ["kernels.cu", "lbmp_api.cu", "noalloc.cu", "batch.cu", "adjoint.cu"]
HEADERS = ["lattice.cuh", "kernels.h", "staged.cuh", "wide.cuh", "context.h", "nvtx_range.h", "device_scope.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
              "-Xptxas", "-O3", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbmp")
    return cand


def source_hash() -> str:
    """Hash of every source file of the library (kernel identity)."""
    h = hashlib.sha256()
    for name in SOURCES + HEADERS:
        with open(os.path.join(CSRC, name), "rb") as fh:
            h.update(name.encode() + b"\0" + fh.read())
    with open(os.path.join(ROOT, "include", "lbmp.h"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


STEP_KERNEL_FILES = ["kernels.cu", "kernels.h", "lattice.cuh", "staged.cuh"]
ADJOINT_KERNEL_FILES = ["adjoint.cu", "kernels.h", "lattice.cuh"]
BATCH_KERNEL_FILES = ["batch.cu", "kernels.h", "lattice.cuh", "staged.cuh"]


def kernel_hash(files=STEP_KERNEL_FILES) -> str:
    """Hash of the files that define a group of kernels (the time-step
    kernels by default): the identity of the kernels whose DRAM traffic the
    committed ncu summaries record."""
    h = hashlib.sha256()
    for name in files:
        with open(os.path.join(CSRC, name), "rb") as fh:
            h.update(name.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def _stamp() -> str:
    return os.path.join(OUT_DIR, "liblbmp.hash")


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(_stamp()):
        return False
    with open(_stamp()) as fh:
        return fh.read().strip() == source_hash() + " " + os.uname().machine


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []

    def compile_one(name):
        obj = os.path.join(OUT_DIR, name.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, *inc, "-c", os.path.join(CSRC, name), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    objs = [o for o, _ in results]
    if verbose or ptxas_verbose:
        for _, log in results:
            sys.stdout.write(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of liblbmp failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(_stamp(), "w") as fh:
        fh.write(source_hash() + " " + os.uname().machine)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_verbose="-v" in sys.argv))
