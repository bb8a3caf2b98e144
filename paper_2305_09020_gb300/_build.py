"""Compile the in-tree CUDA library ``libpf.so`` for sm_103a with nvcc (no cmake)."""
from __future__ import annotations

import hashlib
import os
import subprocess
import tempfile

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "libpf.so")
SOURCES = ["pf_api.cu", "pf_setup.cpp", "pf_static.cu", "pf_no.cu", "pf_peaks.cu"]
HEADERS = ["pf_kernels.cuh", "pf_tc.cuh"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _digest() -> str:
    h = hashlib.sha256()
    for f in SOURCES + HEADERS:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(ROOT, "include", "pf.h"), "rb") as fh:
        h.update(fh.read())
    h.update(ARCH.encode())
    return h.hexdigest()


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Build libpf.so next to this file unless an up-to-date copy exists."""
    stamp = LIB + ".sha256"
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == dig:
                return LIB
    tmp = LIB + ".tmp"
    flags = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off"]
    with tempfile.TemporaryDirectory(prefix="pf_build_") as work:
        # one nvcc per translation unit, all at once, then one link
        objs, procs = [], []
        for f in SOURCES:
            obj = os.path.join(work, f + ".o")
            cmd = [nvcc(), *flags, "-c", os.path.join(CSRC, f), "-o", obj]
            if verbose:
                print(" ".join(cmd))
            procs.append((cmd, subprocess.Popen(cmd)))
            objs.append(obj)
        for cmd, p in procs:
            if p.wait() != 0:
                raise subprocess.CalledProcessError(p.returncode, cmd)
        subprocess.run([nvcc(), ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return LIB
