"""Build libpsc.so in place (nvcc, sm_103a only), and libpsc_debug.so, the
bounds-checked debug build (PSC_DEBUG=1: every indexed access on the hot path
checks its index, records the first violation and stays in bounds; the call
that launched the kernel then fails with PSC_EDEVICE).

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
LIB_DEBUG = os.path.join(HERE, "libpsc_debug.so")
OBJ = os.path.join(HERE, "_obj")
OBJ_DEBUG = os.path.join(HERE, "_obj_debug")
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


def _flags(src, verbose, debug=False):
    f = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
         "-I", os.path.join(ROOT, "include")]
    if os.path.basename(src) in FAST_MATH:
        f.append("--use_fast_math")
    if debug:
        f.append("-DPSC_DEBUG=1")
    if verbose:
        f.append("-Xptxas=-v")
    return f


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _inputs())


def build(force: bool = False, verbose: bool = False, debug: bool = None) -> str:
    """Compile every CUDA source of the package into libpsc.so (in place);
    debug=True builds only libpsc_debug.so, debug=None (default) both, in one
    pool of compiler processes.  Returns the release library's path (the
    debug one's for debug=True)."""
    variants = [False, True] if debug is None else [bool(debug)]
    todo = [v for v in variants if force or _stale(LIB_DEBUG if v else LIB)]
    if todo:
        exe = nvcc()
        for v in todo:
            os.makedirs(OBJ_DEBUG if v else OBJ, exist_ok=True)

        def compile_one(job):
            src, v = job
            obj = os.path.join(OBJ_DEBUG if v else OBJ, os.path.basename(src) + ".o")
            subprocess.check_call([exe, *_flags(src, verbose, v), "-c", "-o", obj, src], cwd=HERE)
            return obj

        jobs = [(src, v) for v in todo for src in sources()]
        with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            objs = list(ex.map(compile_one, jobs))
        for v in todo:
            lib = LIB_DEBUG if v else LIB
            mine = [o for o, (_, jv) in zip(objs, jobs) if jv == v]
            subprocess.check_call([exe, *ARCH, "-shared", "-o", lib + ".tmp", *mine], cwd=HERE)
            os.replace(lib + ".tmp", lib)
    return LIB_DEBUG if debug else LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
