"""Build the library's shared object (libmpt.so) in-tree with nvcc for sm_103a.

Each translation unit compiles in parallel, then one link step; no CMake.  Run as
``python -m paper_2604_22228_gb300.build`` or call ``build()``.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "libmpt.so")
OBJDIR = os.path.join(PKG, "_build")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
SOURCES = ["copy_kernels.cu", "copy_bulk.cu", "stage_consume.cu", "runtime.cu", "planner.cpp", "api_plan.cpp", "model.cpp", "tuner.cu", "batch.cu", "serve.cu", "jacobi.cu", "noalloc.cu", "host_pool.cpp", "host_probe.cpp"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmpt.so")


CFLAGS = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3,-fvisibility=hidden"]
HEADERS = ["kernels.cuh", "bulk_config.h", "batch_kernels.cuh", "copy_device.cuh", "internal.h", "ctx.h", "host_pool.h"]
STAMP = OUT + ".sha256"


def _compile(nvcc: str, src: str) -> str:
    obj = os.path.join(OBJDIR, os.path.basename(src) + ".o")
    cmd = [nvcc] + CFLAGS + ["-I", INCLUDE, "-I", CSRC, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def source_hash(nvcc: str | None = None) -> str:
    """sha256 over every source and header the library is built from (names and bytes), the
    compile flags, the machine type and the nvcc in use: the key under which a built
    libmpt.so may be reused."""
    import hashlib
    import platform
    h = hashlib.sha256()
    files = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(INCLUDE, "mpt.h")]
    for f in files:
        h.update(os.path.relpath(f, ROOT).encode() + b"\0")
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(CFLAGS).encode())
    h.update(platform.machine().encode())
    h.update((nvcc or "").encode())
    return h.hexdigest()


def build(force: bool = False) -> str:
    """Compile every source and link libmpt.so; returns its path.  An existing libmpt.so is
    reused only when the stamp written beside it at link time holds the current
    source_hash(); anything else (edited sources or flags, another machine type, a library
    copied in from elsewhere without its stamp) rebuilds."""
    nvcc = _nvcc()
    key = source_hash(nvcc)
    if not force and os.path.exists(OUT) and os.path.exists(STAMP):
        with open(STAMP) as f:
            if f.read().strip() == key:
                return OUT
    os.makedirs(OBJDIR, exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s), SOURCES))
    tmp = OUT + ".tmp"
    cmd = [nvcc, ARCH, "-shared", "-o", tmp] + objs + ["-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    if os.path.exists(STAMP):
        os.unlink(STAMP)
    os.replace(tmp, OUT)
    with open(STAMP + ".tmp", "w") as f:
        f.write(key + "\n")
    os.replace(STAMP + ".tmp", STAMP)
    return OUT


if __name__ == "__main__":
    print(build(force=True))
