"""Build the CUDA library libhpse.so in-tree for sm_103a (GB300).

Generates one translation unit per (precision, degree W = 1..HPSE_MAX_W) from
csrc/inst_template.cuh, compiles every unit with nvcc in parallel and links
them with the host library csrc/hpse.cu into paper_1110_2316_gb300/libhpse.so.
Only nvcc is needed (no CMake, no torch extension machinery).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
GEN = os.path.join(BUILD, "gen")
LIB = os.path.join(PKG, "libhpse.so")
MAX_W = 10
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhpse.so")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC] + list(extra)


def _generate():
    os.makedirs(GEN, exist_ok=True)
    units = []
    for prec, real, extra in (("f64", "double", "#define HPSE_DOUBLE\n"), ("f32", "float", "")):
        for w in range(1, MAX_W + 1):
            path = os.path.join(GEN, f"inst_{prec}_w{w}.cu")
            text = (f"#define REAL {real}\n#define WDEG {w}\n"
                    f"#define HPSE_REGISTER_NAME hpse_register_{prec}_w{w}\n{extra}"
                    f'#include "inst_template.cuh"\n')
            if not os.path.exists(path) or open(path).read() != text:
                with open(path, "w") as f:
                    f.write(text)
            units.append(path)
    units.append(os.path.join(CSRC, "hpse.cu"))
    return units


def _deps_mtime():
    m = 0.0
    for d in (CSRC, os.path.join(ROOT, "include")):
        for fn in os.listdir(d):
            m = max(m, os.path.getmtime(os.path.join(d, fn)))
    return m


def build(verbose: bool = False, jobs: int | None = None) -> str:
    """Compile (incrementally) and link libhpse.so; returns its path."""
    cc = nvcc()
    units = _generate()
    dep_m = _deps_mtime()
    objs = []
    todo = []
    for u in units:
        o = os.path.join(BUILD, os.path.basename(u)[:-3] + ".o")
        objs.append(o)
        if not os.path.exists(o) or os.path.getmtime(o) < max(dep_m, os.path.getmtime(u)):
            todo.append((u, o))

    def compile_one(uo):
        u, o = uo
        cmd = [cc] + _flags() + ["-c", u, "-o", o + ".tmp"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (u, res.stdout, res.stderr))
        os.replace(o + ".tmp", o)
        if verbose:
            sys.stdout.write("compiled %s\n" % os.path.basename(u))
        return o

    if todo:
        n = jobs or max(1, min(len(todo), os.cpu_count() or 4))
        with ThreadPoolExecutor(n) as ex:
            list(ex.map(compile_one, todo))
    if todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [cc] + ARCH + ["-shared", "-cudart", "shared", "-o", LIB + ".tmp"] + objs + \
              ["-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (res.stdout, res.stderr))
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
