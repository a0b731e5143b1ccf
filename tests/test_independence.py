"""The oracle and the CUDA path share no code: no Python import, C include or library
reference crosses between `oracle/` and the package, except the package's input generators
(`workloads.py`, configuration and random numbers only), which both may read."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2607_13740_b300")
ORC = os.path.join(ROOT, "oracle")


def _read(p):
    with open(p, encoding="utf-8") as f:
        return f.read()


def test_package_never_imports_or_links_the_oracle():
    for p in glob.glob(os.path.join(PKG, "*.py")) + glob.glob(os.path.join(PKG, "csrc", "*")):
        src = _read(p)
        assert not re.search(r"^\s*(from|import)\s+oracle\b", src, re.M), p
        assert "grace_oracle" not in src, p
        assert not re.search(r'#include\s+"[^"]*oracle', src), p


def test_oracle_never_imports_or_links_the_cuda_path():
    for p in glob.glob(os.path.join(ORC, "*.py")) + glob.glob(os.path.join(ORC, "*.c")) + \
            glob.glob(os.path.join(ORC, "*.h")):
        src = _read(p)
        for m in re.finditer(r"^\s*(?:from|import)\s+([\w.]+)", src, re.M):
            mod = m.group(1)
            assert not mod.startswith("paper_2607_13740_b300") or mod.endswith("workloads"), (p, mod)
        assert "libgrace.so" not in src and "grace.h" not in src and "csrc" not in src, p


def test_workloads_hold_no_method_arithmetic():
    """The shared input module neither imports numerical kernels nor defines the scheme's
    operators: it holds configuration and seeded random numbers."""
    src = _read(os.path.join(PKG, "workloads.py"))
    for word in ("legendre", "legval", "gauss", "quad(", "limiter_gamma", "np.linalg"):
        assert word not in src.lower(), word
