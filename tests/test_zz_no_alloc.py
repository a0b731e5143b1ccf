"""grace_rhs_noalloc: the RHS entry point that allocates nothing.

It is for callers that cannot allocate device memory (a host framework that
owns all device memory through its own pool, or a per-substep loop where the
device synchronisation of cudaMalloc is not acceptable).  Its output must
match grace_rhs on the same inputs, on consecutive calls that reuse the
library's fixed workspace.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2607_13740_b300 import grace, workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _noalloc():
    L = grace.load()
    f = L.grace_rhs_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _scaled(L, Lo, S):
    den = np.maximum(np.abs(Lo), S)
    d = np.abs(L - Lo)
    return np.where(den > 0, d / np.where(den > 0, den, 1.0), np.where(d > 0, np.inf, 0.0))


def test_noalloc_rhs_matches_grace_rhs_on_consecutive_calls():
    spec = W.additive_spec(40, 2)
    ctx = grace.Context([spec])
    f = _noalloc()
    for call, (n, seed) in enumerate([(300, 501), (131, 502)]):
        g = torch.as_tensor(W.random_coefficients(spec, n, seed=seed), device=DEV)
        ref = ctx.batch(n).rhs(g)
        out = torch.full_like(g, float("nan"))
        ctx.set_stream()
        st = f(ctx._h, 0, n, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        assert st == 0, grace.load().grace_last_error().decode()
        torch.cuda.synchronize()
        a, r = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(a).all()
        Lo, S = oracle.Oracle(spec).rhs(g.cpu().numpy())
        assert _scaled(a, Lo, S).max() <= 1e-12, call
        assert _scaled(a, r, S).max() <= 1e-12, call


def test_noalloc_rejects_sizes_beyond_the_fixed_workspace():
    spec = W.additive_spec(40, 2)
    ctx = grace.Context([spec])
    P, R = ctx.group_info(0)
    too_many = (2 ** 21) // R + 1
    # buffers of the full size, so that a regressed size guard computes wrong values instead of
    # reading or writing past an allocation
    g = torch.zeros(too_many * P, dtype=torch.float64, device=DEV)
    out = torch.zeros_like(g)
    st = _noalloc()(ctx._h, 0, too_many, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(out.data_ptr()))
    torch.cuda.synchronize()
    assert st == 1
    assert "exceeds" in grace.load().grace_last_error().decode()
