"""Compile libepic.so (the CUDA kernels and the C ABI) for sm_103a, in tree.

Every translation unit under csrc/ is compiled in parallel with nvcc, then
linked into ``paper_1904_11422_gb300/libepic.so`` (CUDA runtime linked
statically).  Objects go to ``paper_1904_11422_gb300/_build/``.  The library
is rebuilt whenever the hash of its sources, headers, flags, compiler version
and host architecture differs from the one recorded beside the objects, so a
library copied from another machine or built from other sources is never
reused.
"""
from __future__ import annotations

import glob
import hashlib
import os
import platform
import shutil
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libepic.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(verbose_ptxas: bool) -> list[str]:
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "-Xcompiler", "-Wall", "--expt-relaxed-constexpr"] + ARCH
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


_NVCC_VERSION: list[str] = []


def _stamp() -> str:
    """Hash of everything the library is built from: every source and header,
    the public header, the compiler flags, the nvcc version and the host
    architecture."""
    h = hashlib.sha256()
    deps = sorted(sources() + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(HERE, "..", "include", "*.h")))
    for d in deps:
        h.update(os.path.basename(d).encode())
        with open(d, "rb") as f:
            h.update(f.read())
    h.update(" ".join(_flags(False) + ARCH).encode())
    if not _NVCC_VERSION:
        _NVCC_VERSION.append(subprocess.run([nvcc(), "--version"], capture_output=True, text=True).stdout)
    h.update(_NVCC_VERSION[0].encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


STAMP = os.path.join(BUILD, "libepic.stamp")


def _stale(stamp: str) -> bool:
    if not os.path.exists(LIB) or not os.path.exists(STAMP):
        return True
    with open(STAMP) as f:
        return f.read().strip() != stamp


def build(force: bool = False, verbose_ptxas: bool = False, quiet: bool = True) -> str:
    stamp = _stamp()
    if not force and not _stale(stamp):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    t0 = time.time()
    procs = []
    objs = []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [nvcc()] + _flags(verbose_ptxas) + ["-c", src, "-o", obj]
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = []
    for src, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            failed.append((src, out))
        elif out and (verbose_ptxas or not quiet):
            sys.stderr.write(out)
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    tmp = LIB + f".{os.getpid()}.tmp"
    link = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}")
    os.replace(tmp, LIB)
    with open(STAMP + f".{os.getpid()}.tmp", "w") as f:
        f.write(stamp + "\n")
    os.replace(STAMP + f".{os.getpid()}.tmp", STAMP)
    if not quiet:
        sys.stderr.write(f"libepic.so built in {time.time() - t0:.1f}s\n")
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, quiet=False)
