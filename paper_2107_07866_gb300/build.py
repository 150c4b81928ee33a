"""Builds the CUDA library (libmisa.so) in-tree for sm_103a with nvcc.

One translation unit (host runtime + kernels, FP32 and FP64 instantiations);
``python -m paper_2107_07866_gb300.build`` or ``build()``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "libmisa.so")
SOURCES = [os.path.join(PKG, "csrc", "misa_api.cu")]
DEPS = SOURCES + sorted(os.path.join(PKG, "csrc", f) for f in os.listdir(os.path.join(PKG, "csrc"))
                        if f.endswith(".cuh")) + [os.path.join(ROOT, "include", "misa.h")]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmisa.so")


def command(out=LIB, extra=()):
    return [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
            "-I" + os.path.join(ROOT, "include"), "-o", out, *SOURCES, *extra]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    tmp = LIB + ".tmp"
    cmd = command(tmp)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    if verbose:
        sys.stdout.write(r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
