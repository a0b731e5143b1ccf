"""grace_step_host: the state and time steps in host memory, copies inside the call.

Its results must equal grace_step on device buffers bit for bit (same kernels); successive
calls on page-locked buffers overlap through double-buffered staging and must still give
every call its own result."""
import numpy as np
import pytest
import torch

from paper_2607_13740_b300 import grace, workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
FORMS = [grace.FP64, grace.TF32, grace.BF16X3]
IDS = ["fp64", "tf32", "bf16x3"]


def _device_step(b, g0, dt, n_steps, form):
    g = g0.to(DEV)
    mass = torch.zeros(b.n_cells, dtype=torch.float64, device=DEV)
    flags = torch.zeros(b.n_cells, dtype=torch.uint8, device=DEV)
    b.step(g, dt.to(DEV), n_steps, form, mass=mass, flags=flags)
    torch.cuda.synchronize()
    return g.cpu(), mass.cpu(), flags.cpu()


@pytest.mark.parametrize("form", FORMS, ids=IDS)
def test_host_step_equals_device_step(form):
    """300 cells (two 128-cell tiles and a ragged tail), 3 steps, pinned buffers."""
    wl = W.batched_additive(n_cells=300)
    ctx = grace.Context([wl.spec], 0, precisions=(grace.FP64, grace.TF32, grace.BF16X3))
    b = ctx.batch(wl.n_cells)
    g0 = b.project(wl.ic_kind, wl.ic_params).cpu()
    dt = torch.as_tensor(wl.dt, dtype=torch.float64)
    ref = _device_step(b, g0, dt, 3, form)
    h_in, h_dt = g0.pin_memory(), dt.pin_memory()
    h_out = torch.empty_like(g0).pin_memory()
    mass = torch.zeros(b.n_cells, dtype=torch.float64).pin_memory()
    flags = torch.zeros(b.n_cells, dtype=torch.uint8).pin_memory()
    b.step_host(h_in, h_dt, 3, form, out=h_out, mass=mass, flags=flags)
    b.wait_host()
    assert b.device_error() == 0
    assert torch.equal(h_out, ref[0]) and torch.equal(mass, ref[1]) and torch.equal(flags, ref[2])
    np.testing.assert_array_equal(h_in.numpy(), g0.numpy())      # the input is left unchanged


def test_pipelined_calls_keep_their_own_results():
    """Five successive calls (two staging slots) with different inputs and outputs, waited
    once at the end, each equal to its own device step; then in place on pageable memory."""
    wl = W.batched_additive(n_cells=1000)
    ctx = grace.Context([wl.spec], 0, precisions=(grace.FP64, grace.BF16X3))
    b = ctx.batch(wl.n_cells)
    g0 = b.project(wl.ic_kind, wl.ic_params).cpu()
    dt = torch.as_tensor(wl.dt, dtype=torch.float64)
    inputs = [(g0 * (1.0 + 0.25 * i)).pin_memory() for i in range(5)]
    outs = [torch.empty_like(g0).pin_memory() for _ in range(5)]
    h_dt = dt.pin_memory()
    for i in range(5):
        b.step_host(inputs[i], h_dt, 2, grace.BF16X3, out=outs[i])
    b.wait_host()
    for i in range(5):
        ref, _, _ = _device_step(b, inputs[i], dt, 2, grace.BF16X3)
        assert torch.equal(outs[i], ref), i
    pageable = g0.clone()
    b.step_host(pageable, dt.clone(), 2, grace.BF16X3)
    b.wait_host()
    ref, _, _ = _device_step(b, g0, dt, 2, grace.BF16X3)
    assert torch.equal(pageable, ref)


@pytest.mark.parametrize("form", [grace.FP64, grace.BF16X3], ids=["fp64", "bf16x3"])
def test_pinned_chained_and_in_place_calls_need_no_waits(form):
    """Page-locked buffers, no wait between calls: (a) a chain where each call reads the
    previous call's output (h_g of call i = h_out of call i-1), (b) five in-place calls on one
    buffer.  The upload of a call that reads what the previous call writes must follow that
    call's download; every result equals the device-step chain bit for bit."""
    wl = W.batched_additive(n_cells=1000)
    ctx = grace.Context([wl.spec], 0, precisions=(grace.FP64, form))
    b = ctx.batch(wl.n_cells)
    g0 = b.project(wl.ic_kind, wl.ic_params).cpu()
    dt = torch.as_tensor(wl.dt, dtype=torch.float64)
    refs = [g0]
    for i in range(5):
        refs.append(_device_step(b, refs[-1], dt, 2, form)[0])
    h_dt = dt.pin_memory()
    bufs = [g0.pin_memory()] + [torch.full_like(g0, float("nan")).pin_memory() for _ in range(5)]
    for i in range(5):
        b.step_host(bufs[i], h_dt, 2, form, out=bufs[i + 1])
    b.wait_host()
    for i in range(1, 6):
        assert torch.equal(bufs[i], refs[i]), i
    inplace = g0.pin_memory()
    for i in range(5):
        b.step_host(inplace, h_dt, 2, form)
    b.wait_host()
    assert b.device_error() == 0
    assert torch.equal(inplace, refs[5])


def test_mixed_group_batch_and_graph_replay():
    """A batch mixing groups of several N and k (grouped tensor step), then the same batch
    with graph replay on a bound non-default stream (one staging slot)."""
    specs, group, ic, dt = W.uneven_batch(400, seed=1108, n_range=(8, 14), orders=(0, 1, 2, 3))
    ctx = grace.Context(specs, 0, precisions=(grace.FP64, grace.BF16X3))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = ctx.batch(len(group), group)
        g0 = b.project(W.IC_EXP, ic).cpu()
        dtt = torch.as_tensor(dt, dtype=torch.float64)
        ref, _, _ = _device_step(b, g0, dtt, 2, grace.BF16X3)
        out = torch.empty_like(g0).pin_memory()
        h_in, h_dt = g0.pin_memory(), dtt.pin_memory()
        b.step_host(h_in, h_dt, 2, grace.BF16X3, out=out)
        b.wait_host()
        assert torch.equal(out, ref)
        b.set_graph(True)
        for _ in range(3):
            out.zero_()
            b.step_host(h_in, h_dt, 2, grace.BF16X3, out=out)
            b.wait_host()
            assert torch.equal(out, ref)


def test_host_step_rejects_device_tensors():
    wl = W.batched_additive(n_cells=8)
    ctx = grace.Context([wl.spec], 0)
    b = ctx.batch(8)
    g = b.project(wl.ic_kind, wl.ic_params)
    with pytest.raises(grace.GraceError):
        b.step_host(g, torch.zeros(8, dtype=torch.float64), 1)
