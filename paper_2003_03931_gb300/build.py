"""Build libpmpm.so in-tree with nvcc for sm_103a (GB300).

Compiles each CUDA translation unit in parallel and links a shared library
next to this file.  Used by ``__graft_entry__.build()``; runs without a GPU.
"""

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpmpm.so")
UNITS = ["abi.cu", "green.cu", "fft.cu", "coarse.cu", "tile.cu", "sort.cu", "ic.cu", "power.cu", "serve.cu",
         "noalloc.cu", "probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libpmpm")
    return path


def _compile(unit, verbose, build_dir, defines):
    src = os.path.join(SRC, unit)
    obj = os.path.join(build_dir, unit.replace(".cu", ".o"))
    cmd = [nvcc(), *ARCH, *FLAGS, *["-D" + d for d in defines], "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {unit}:\n{r.stderr}")
    return obj, r.stderr


def build(verbose=False, force=False, defines=(), lib=None, build_dir=None):
    """Build libpmpm.so (or, with ``lib``/``build_dir``, a variant compiled
    with extra preprocessor ``defines``); returns the library path."""
    lib = lib or LIB
    build_dir = build_dir or BUILD
    os.makedirs(build_dir, exist_ok=True)
    sources = [os.path.join(SRC, u) for u in UNITS]
    headers = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith(".cuh")]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "pmpm.h"))
    if not force and os.path.exists(lib):
        newest = max(os.path.getmtime(p) for p in sources + headers + [__file__])
        if os.path.getmtime(lib) >= newest:
            return lib
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(lambda u: _compile(u, verbose, build_dir, defines), UNITS))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
