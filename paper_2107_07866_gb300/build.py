"""Builds the CUDA library (libmisa.so) in-tree for sm_103a with nvcc.

Six translation units compiled in parallel and linked into one shared
library: the host runtime with the MD, adjoint and per-site alloy kernels
(``misa_api.cu``), the FP32 tile gathers split by tile shape over three
units (``misa_tiles_f32_{a,b,c}.cu``), the FP64 tile gathers
(``misa_tiles_f64.cu``) and the issue-rate microbenchmarks
(``misa_probe.cu``).  ``python -m
paper_2107_07866_gb300.build`` or ``build()``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "libmisa.so")
OBJDIR = os.path.join(PKG, "_build")
SOURCES = [os.path.join(PKG, "csrc", f) for f in ("misa_tiles_f32_a.cu", "misa_tiles_f32_b.cu", "misa_tiles_f32_c.cu",
                                                   "misa_api.cu", "misa_tiles_f64.cu", "misa_probe.cu")]
DEPS = SOURCES + sorted(os.path.join(PKG, "csrc", f) for f in os.listdir(os.path.join(PKG, "csrc"))
                        if f.endswith(".cuh")) + [os.path.join(ROOT, "include", "misa.h")]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmisa.so")


def compile_command(src: str, obj: str, extra=()) -> list:
    return [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
            "-I" + os.path.join(ROOT, "include"), "-c", src, "-o", obj, *extra]


def link_command(objs, out: str) -> list:
    return [nvcc(), ARCH, "-shared", "-o", out, *objs]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    objs = [os.path.join(OBJDIR, os.path.splitext(os.path.basename(s))[0] + ".o") for s in SOURCES]
    cmds = [compile_command(s, o) for s, o in zip(SOURCES, objs)]
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
    outs = [p.communicate()[0] for p in procs]
    for c, p, o in zip(cmds, procs, outs):
        if p.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(c) + "\n" + o)
        if verbose:
            sys.stdout.write(o)
    tmp = LIB + ".tmp"
    cmd = link_command(objs, tmp)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
