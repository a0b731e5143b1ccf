"""Failure detection of the tensor-core contraction, without a GPU fault.

Every mbarrier wait of the tcgen05 kernels is bounded.  grace_test_arm_wait_timeout makes the
next contraction launch withhold its operand copies, so its MMA issuer waits on a barrier that
nothing arrives at; with a limit of about a millisecond the wait gives up, the kernel records the
failure in the batch's device error word, drains, frees its tensor memory and returns.  The test
checks the status the host reads and that the context stays usable.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_13740_b300 import grace, workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _scaled(L, Lo, S):
    den = np.maximum(np.abs(Lo), S)
    d = np.abs(L - Lo)
    return np.where(den > 0, d / np.where(den > 0, den, 1.0), np.where(d > 0, np.inf, 0.0))


@pytest.mark.parametrize("form", [grace.TF32, grace.BF16X3], ids=["tf32", "bf16x3"])
def test_bounded_wait_runs_out_and_reports_timeout(form):
    spec = W.additive_spec(12, 2, 1e-3, 1e4)
    ctx = grace.Context([spec], 0, precisions=(grace.FP64, form))
    n = 300
    b = ctx.batch(n)
    g = torch.as_tensor(W.random_coefficients(spec, n, seed=41), device=DEV)
    assert b.device_error() == 0
    grace.arm_wait_timeout(2_000_000)          # about 1 ms at 2 GHz
    b.rhs(g, form)                              # returns at once; the launch aborts on the device
    code = b.device_error()                     # synchronises, reads and clears the word
    assert code != 0
    assert b.device_error() == 0                # cleared
    # the context and the batch stay usable: the next call is normal and matches the oracle
    L = b.rhs(g, form).cpu().numpy()
    assert b.device_error() == 0
    Lo, S = oracle.Oracle(spec).rhs(g.cpu().numpy())
    tol = {grace.TF32: 2e-3, grace.BF16X3: 5e-5}[form]
    assert _scaled(L, Lo, S).max() <= tol

