"""In-tree build of the CUDA library ``_build/libmapsmoother.so`` for sm_103a.

Each solver instance is its own translation unit (one nvcc process per
(model, nx, ny, precision)), compiled in parallel, then linked into one shared
library with the static CUDA runtime.  Objects are reused when they are newer
than every source file and were built with the same flags.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmapsmoother.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]

# (nx, ny) of the linear-model instances; keep in sync with MAP_LINEAR_SHAPES in capi.cu
LINEAR_SHAPES = [(2, 1), (3, 1), (4, 2), (5, 2), (6, 3), (8, 4)]
CUBIC_SHAPES = [(2, 2)]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def units():
    """(object name, source, extra defines) of every translation unit."""
    out = [("capi", "capi.cu", []), ("discretise", "discretise.cu", []), ("noalloc", "noalloc.cu", []),
           ("batch", "batch.cu", []), ("batch_persist", "batch_persist.cu", []),
           ("peaks", "peaks.cu", []), ("selftest", "selftest.cu", [])]
    for prec, typ in (("f32", "float"), ("f64", "double")):
        for n, m in LINEAR_SHAPES:
            for part in ((0, 1) if n <= 6 else (0,)):
                out.append((f"lin_{n}_{m}_{prec}_{part}", "inst_linear.cu",
                            [f"-DINST_N={n}", f"-DINST_M={m}", f"-DINST_S={typ}", f"-DINST_PART={part}"]))
        out.append((f"ct_{prec}", "inst_nonlinear.cu", ["-DINST_CT=1", f"-DINST_S={typ}"]))
        for n, m in CUBIC_SHAPES:
            out.append((f"cubic_{n}_{m}_{prec}", "inst_nonlinear.cu",
                        ["-DINST_CT=0", f"-DINST_N={n}", f"-DINST_M={m}", f"-DINST_S={typ}"]))
    return [u for u in out if os.path.exists(os.path.join(CSRC, u[1]))]


def _newest_source() -> float:
    newest = 0.0
    for root in (CSRC, os.path.join(os.path.dirname(HERE), "include")):
        for f in os.listdir(root):
            newest = max(newest, os.path.getmtime(os.path.join(root, f)))
    return newest


def _compile(args):
    cmd, obj, stamp, sig = args
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        return obj, r.stdout + r.stderr
    with open(stamp, "w") as f:
        f.write(sig)
    return obj, None


def build(jobs: int | None = None, verbose: bool = False) -> str:
    """Compile every translation unit that is out of date and link the library."""
    os.makedirs(BUILD, exist_ok=True)
    newest = _newest_source()
    todo, objs = [], []
    for name, src, defs in units():
        obj = os.path.join(BUILD, name + ".o")
        stamp = obj + ".sig"
        cmd = [nvcc(), *ARCH, *FLAGS, *defs, "-c", os.path.join(CSRC, src), "-o", obj]
        sig = hashlib.sha1(" ".join(cmd).encode()).hexdigest()
        objs.append(obj)
        fresh = (os.path.exists(obj) and os.path.getmtime(obj) >= newest and os.path.exists(stamp)
                 and open(stamp).read() == sig)
        if not fresh:
            todo.append((cmd, obj, stamp, sig))
    if todo:
        jobs = jobs or max(1, min(len(todo), os.cpu_count() or 4))
        with ThreadPoolExecutor(jobs) as ex:
            for obj, err in ex.map(_compile, todo):
                if verbose:
                    print("built", os.path.basename(obj), file=sys.stderr)
                if err:
                    raise RuntimeError(f"nvcc failed for {obj}:\n{err}")
    if todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static",
                               "-Xlinker", "--no-undefined"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
