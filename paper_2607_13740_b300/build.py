"""Builds the CUDA C-ABI library paper_2607_13740_b300/libgrace.so for sm_103a (in-tree).

Run as ``python -m paper_2607_13740_b300.build`` or through ``__graft_entry__.build()``.
nvcc cross-compiles without a GPU.  Every translation unit compiles to its own object under
``_build/`` (in parallel; only the stale ones), then one link step writes the library.
"""
import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libgrace.so")
OBJ = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def _headers():
    return glob.glob(os.path.join(HERE, "csrc", "*.h")) + glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + \
        [os.path.join(ROOT, "include", "grace.h")]


def _obj(src):
    return os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _nvcc():
    return os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _compile(src, verbose):
    cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-c", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-fvisibility=hidden", "-I", os.path.join(ROOT, "include"),
           "--expt-relaxed-constexpr", "-o", _obj(src) + ".tmp", src]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(_obj(src) + ".tmp", _obj(src))


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    srcs = sources()
    hdrs = _headers()
    todo = [s for s in srcs if force or verbose or _stale(_obj(s), [s] + hdrs)]
    if todo:
        with ThreadPoolExecutor(max_workers=max(1, min(len(todo), os.cpu_count() or 1))) as ex:
            for f in [ex.submit(_compile, s, verbose) for s in todo]:
                f.result()
    objs = [_obj(s) for s in srcs]
    if force or todo or _stale(LIB, objs):
        subprocess.run([_nvcc(), *ARCH, "-shared", "-o", LIB + ".tmp", *objs], check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
