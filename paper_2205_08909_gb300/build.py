"""Builds the CUDA library libmfcg.so in-tree for sm_103a.

Every translation unit under csrc/ is compiled in parallel with nvcc and the
objects are linked into paper_2205_08909_gb300/_lib/libmfcg.so.  Nothing is
installed elsewhere.
"""
from __future__ import annotations

import concurrent.futures
import glob
import hashlib
import os
import platform
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "_lib")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(LIBDIR, "libmfcg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmfcg.so")


def _sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    deps = _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
    deps.append(os.path.join(PKG, "..", "include", "mfcg.h"))
    return sorted(os.path.abspath(d) for d in deps if os.path.exists(d))


def _source_hash() -> str:
    """SHA-256 over the compiler flags and the name and content of every source
    and header: the library is rebuilt whenever it differs from the hash stored
    beside it, whatever the files' modification times (a library copied in with
    the tree is never trusted)."""
    h = hashlib.sha256()
    h.update(" ".join(ARCH + FLAGS).encode())
    for d in _deps():
        h.update(os.path.relpath(d, PKG).encode())
        with open(d, "rb") as fh:
            h.update(fh.read())
    h.update(platform.machine().encode())
    return h.hexdigest()


STAMP = LIB + ".sha256"


def _up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(STAMP):
        return False
    with open(STAMP) as fh:
        return fh.read().strip() == _source_hash()


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and _up_to_date():
        return LIB
    nvcc = _nvcc()
    if os.path.exists(STAMP):
        os.remove(STAMP)
    os.makedirs(LIBDIR, exist_ok=True)
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stderr}")
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        return obj

    workers = min(len(_sources()), os.cpu_count() or 4)
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as fh:
        fh.write(_source_hash() + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
