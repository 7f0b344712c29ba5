"""Builds the in-tree shared library ``_build/libqtn.so`` for sm_103a.

Host sources (network, planning, step programs) and CUDA sources (kernels,
C-ABI layer) are compiled in parallel by nvcc and linked into one library.
"""
from __future__ import annotations

import concurrent.futures
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libqtn.so")

SOURCES = ["network.cpp", "plan.cpp", "program.cpp", "surrogate.cpp", "kernels.cu", "api.cu", "noalloc.cu", "mlp.cu",
           "peaks.cu", "jit.cpp", "wide.cu", "wide_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", BUILD]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _headers_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".hpp", ".cuh", ".h"))]
    paths.append(os.path.join(ROOT, "include", "qtn.h"))
    return max(os.path.getmtime(p) for p in paths)


def _compile(src: str) -> str:
    obj = os.path.join(BUILD, src + ".o")
    path = os.path.join(CSRC, src)
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(path), _headers_mtime()):
        return obj
    cmd = [_nvcc(), *ARCH, *COMMON, "-c", path, "-o", obj + ".tmp"]
    if src.endswith(".cu"):
        cmd[1:1] = ["-lineinfo", "-Xptxas", "-warn-spills"]
    subprocess.run(cmd, check=True)
    os.replace(obj + ".tmp", obj)
    return obj


def _write_arith_source():
    """The shared complex arithmetic (csrc/arith.cuh) as a C++ raw string, for
    the kernels the library generates and compiles at run time."""
    with open(os.path.join(CSRC, "arith.cuh")) as f:
        text = f.read()
    body = 'R"QTNARITH(' + text + ')QTNARITH"\n'
    out = os.path.join(BUILD, "arith_src.inc")
    if not os.path.exists(out) or open(out).read() != body:
        with open(out + ".tmp", "w") as f:
            f.write(body)
        os.replace(out + ".tmp", out)


def build(verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    _write_arith_source()
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.run([_nvcc(), *ARCH, "-shared", "-Xlinker", "-z", "-Xlinker", "defs", "-o", tmp, *objs, "-lcudart",
                        "-ldl"], check=True)
        os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
