"""Build libpsc.so in place (nvcc, sm_103a only).

Each CUDA source is compiled to an object in parallel, then linked.  The
transport kernel is compiled with nvcc's fast FP32 arithmetic (approximate
division and square root, hardware log/exp/sin/cos, denormals flushed);
its parity with the FP64 oracle is tested on exactly this build.  The
finalize and runtime sources keep IEEE FP32 semantics, which the bit-exact
FP64 sensitivity multiply relies on.  No FMA contraction on the host side.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libpsc.so")
OBJ = os.path.join(HERE, "_obj")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FAST_MATH = {"transport.cu"}


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def _inputs():
    return sources() + glob.glob(os.path.join(HERE, "csrc", "*.h*")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h")) + [os.path.abspath(__file__)]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libpsc")
    return exe


def _flags(src, verbose):
    f = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
         "-I", os.path.join(ROOT, "include")]
    if os.path.basename(src) in FAST_MATH:
        f.append("--use_fast_math")
    if verbose:
        f.append("-Xptxas=-v")
    return f


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA source of the package into libpsc.so (in place)."""
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(p) <= t for p in _inputs()):
            return LIB
    os.makedirs(OBJ, exist_ok=True)
    exe = nvcc()

    def compile_one(src):
        obj = os.path.join(OBJ, os.path.basename(src) + ".o")
        subprocess.check_call([exe, *_flags(src, verbose), "-c", "-o", obj, src], cwd=HERE)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, sources()))
    subprocess.check_call([exe, *ARCH, "-shared", "-o", LIB + ".tmp", *objs], cwd=HERE)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
