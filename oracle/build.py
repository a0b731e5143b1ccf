"""Builds the FP64 CPU oracle (test infrastructure) into oracle/libgrace_oracle.so: the oracle
(grace_oracle.c, C), its forward-mode derivative build (grace_oracle_tangent.cpp, the same
source compiled as C++ on dual numbers) and the two-dimensional (mass, volume) oracle
(grace_oracle_mv.c, C).

Run as ``python oracle/build.py`` or through ``__graft_entry__.build()``.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "grace_oracle.c")
SRC_TANGENT = os.path.join(HERE, "grace_oracle_tangent.cpp")
SRC_MV = os.path.join(HERE, "grace_oracle_mv.c")
DUAL_H = os.path.join(HERE, "orc_dual.h")
LIB = os.path.join(HERE, "libgrace_oracle.so")


def build(force: bool = False) -> str:
    newest = max(os.path.getmtime(f) for f in (SRC, SRC_TANGENT, SRC_MV, DUAL_H))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    obj_dir = os.path.join(HERE, "_build")
    os.makedirs(obj_dir, exist_ok=True)
    o_c, o_t = os.path.join(obj_dir, "grace_oracle.o"), os.path.join(obj_dir, "grace_oracle_tangent.o")
    o_mv = os.path.join(obj_dir, "grace_oracle_mv.o")
    warn = ["-Wall", "-Wextra", "-Wno-unused-parameter"]
    subprocess.run(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-fopenmp", *warn, "-c", SRC, "-o", o_c],
                   check=True)
    subprocess.run(["g++", "-O2", "-std=c++17", "-D_GNU_SOURCE", "-fPIC", "-fopenmp", *warn,
                    "-Wno-unused-function", "-Wno-class-memaccess", "-c", SRC_TANGENT, "-o", o_t], check=True)
    subprocess.run(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", *warn, "-c", SRC_MV, "-o", o_mv], check=True)
    tmp = LIB + ".tmp"
    subprocess.run(["g++", "-shared", "-fopenmp", o_c, o_t, o_mv, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
