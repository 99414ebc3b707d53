"""In-tree build of the CUDA library libkrylov_gb300.so for sm_103a.

Compiles every csrc/*.cu translation unit in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a -lineinfo) and links one shared
library into paper_1504_04395_gb300/_lib/.  A content hash of the sources,
the flags and the host architecture is stored next to the library so that an
up-to-date build is reused and a build from another machine is redone.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import platform
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIBNAME = "libkrylov_gb300.so"
LIBPATH = os.path.join(LIBDIR, LIBNAME)

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "-I" + INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkrylov_gb300.so")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def source_digest() -> str:
    """Hash of the CUDA / C sources and compile flags (identifies a kernel build on any host)."""
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode())
                h.update(fh.read())
    h.update(_flags_for_digest().encode())
    return h.hexdigest()


def _flags_for_digest() -> str:
    """The compile flags with the include directory written relative to the repository, so
    that the same sources and flags hash alike on every machine."""
    return " ".join(ARCH_FLAGS + [("-Iinclude" if f == "-I" + INCLUDE else f) for f in NVCC_FLAGS])


def kernel_digest(files) -> str:
    """Hash of the named files under csrc/ and the compile flags (the sources that define one
    kernel and its launch configuration)."""
    h = hashlib.sha256()
    for f in sorted(files):
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    h.update(_flags_for_digest().encode())
    return h.hexdigest()


def _digest() -> str:
    return hashlib.sha256((source_digest() + platform.machine()).encode()).hexdigest()


def _compile(src: str) -> str:
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc()] + ARCH_FLAGS + NVCC_FLAGS + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link the library if its sources changed; returns the library path."""
    stamp = os.path.join(LIBDIR, LIBNAME + ".sha256")
    digest = _digest()
    if not force and os.path.exists(LIBPATH) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == digest:
                return LIBPATH
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    srcs = sources()
    workers = max(1, min(len(srcs), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(_compile, srcs))
    tmp = LIBPATH + ".tmp"
    cmd = [nvcc()] + ARCH_FLAGS + ["-shared", "-o", tmp] + objs + ["-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIBPATH)
    with open(stamp, "w") as fh:
        fh.write(digest)
    if verbose:
        print("built", LIBPATH, file=sys.stderr)
    return LIBPATH


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
