"""Batches mixing groups (different N, k and kernels) and CUDA-graph replay.

A mixed batch must give, cell by cell, exactly the result of running each
group's cells as a separate single-group batch (same kernels, same arithmetic),
and match the oracle at the FP64 parity bar.  Graph replay must reproduce the
direct launches bit for bit, and so must the grouped tensor-form step (one
multi-group contraction and one K-c launch per stage) against the per-group
launch sequences.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2607_13740_b300 import grace, workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
FORMS = (grace.FP64, grace.TF32, grace.BF16X3)


def _mixed(n_cells=300, seed=1104):
    specs, group, ic, dt = W.uneven_batch(n_cells, seed=seed, n_range=(8, 14), orders=(0, 1, 2, 3))
    return specs, group, ic, dt


def _split(arr_flat, offsets, idx):
    return [arr_flat[offsets[c]:offsets[c + 1]] for c in idx]


def test_mixed_rhs_matches_oracle_fp64():
    specs, group, ic, dt = _mixed(120)
    ctx = grace.Context(specs)
    b = ctx.batch(len(group), group)
    off = b.offsets()
    g = b.project(W.IC_EXP, ic)
    L = b.rhs(g).cpu().numpy()
    gh = g.cpu().numpy()
    for gi, spec in enumerate(specs):
        idx = np.where(group == gi)[0]
        if idx.size == 0:
            continue
        o = oracle.Oracle(spec)
        gg = np.stack(_split(gh, off, idx))
        Lo, S = o.rhs(gg)
        Lg = np.stack(_split(L, off, idx))
        den = np.maximum(np.abs(Lo), S)
        err = np.where(den > 0, np.abs(Lg - Lo) / np.where(den > 0, den, 1), np.abs(Lg - Lo) > 0)
        assert err.max() <= 1e-12, (gi, spec)


@pytest.mark.parametrize("form", FORMS, ids=["fp64", "tf32", "bf16x3"])
def test_mixed_step_equals_per_group_batches(form):
    specs, group, ic, dt = _mixed(300)
    ctx = grace.Context(specs, 0, precisions=FORMS)
    b = ctx.batch(len(group), group)
    off = b.offsets()
    g = b.project(W.IC_EXP, ic)
    g0 = g.cpu().numpy()
    dtt = torch.as_tensor(dt, device=DEV)
    mass = torch.zeros(len(group), dtype=torch.float64, device=DEV)
    flags = torch.zeros(len(group), dtype=torch.uint8, device=DEV)
    b.step(g, dtt, 5, form, mass=mass, flags=flags)
    gm = g.cpu().numpy()
    for gi, spec in enumerate(specs):
        idx = np.where(group == gi)[0]
        if idx.size == 0:
            continue
        sb = ctx.batch(idx.size, np.full(idx.size, gi, dtype=np.int32))
        gs = torch.as_tensor(np.stack(_split(g0, off, idx)), device=DEV).contiguous()
        ms = torch.zeros(idx.size, dtype=torch.float64, device=DEV)
        fs = torch.zeros(idx.size, dtype=torch.uint8, device=DEV)
        sb.step(gs.reshape(-1), dtt[idx].contiguous(), 5, form, mass=ms, flags=fs)
        np.testing.assert_array_equal(np.stack(_split(gm, off, idx)), gs.cpu().numpy().reshape(idx.size, -1))
        np.testing.assert_array_equal(mass.cpu().numpy()[idx], ms.cpu().numpy())
        np.testing.assert_array_equal(flags.cpu().numpy()[idx], fs.cpu().numpy())
    assert b.device_error() == 0


def test_mixed_trajectory_matches_oracle_and_conserves_mass():
    specs, group, ic, dt = _mixed(60, seed=1105)
    ctx = grace.Context(specs)
    b = ctx.batch(len(group), group)
    off = b.offsets()
    g = b.project(W.IC_EXP, ic)
    g0 = g.cpu().numpy()
    m0 = b.mass(g).cpu().numpy()
    b.step(g, torch.as_tensor(dt, device=DEV), 10)
    m1 = b.mass(g).cpu().numpy()
    assert np.all(np.abs(m1 - m0) <= 1e-13 * np.abs(m0))
    gg = g.cpu().numpy()
    for gi, spec in enumerate(specs):
        idx = np.where(group == gi)[0]
        if idx.size == 0:
            continue
        go, _, _ = oracle.Oracle(spec).step(np.stack(_split(g0, off, idx)), dt[idx], 10)
        d = np.abs(np.stack(_split(gg, off, idx)) - go)
        assert d.max() <= 1e-10 * np.abs(go).max(), (gi, d.max())


@pytest.mark.parametrize("form", FORMS, ids=["fp64", "tf32", "bf16x3"])
def test_graph_replay_is_bitwise_identical(form):
    specs, group, ic, dt = _mixed(200, seed=1106)
    ctx = grace.Context(specs, 0, precisions=FORMS)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = ctx.batch(len(group), group)
        g = b.project(W.IC_EXP, ic)
        dtt = torch.as_tensor(dt, device=DEV)
        ref = g.clone()
        b.step(ref, dtt, 3, form)
        b.step(ref, dtt, 3, form)
        b.set_graph(True)
        out = g.clone()
        b.step(out, dtt, 3, form)     # captures, then launches
        b.step(out, dtt, 3, form)     # replays
        torch.cuda.synchronize()
    assert torch.equal(out, ref)


@pytest.mark.parametrize("pairs", [grace.CTA_PAIRS_NEVER, grace.CTA_PAIRS_ALWAYS], ids=["single", "pairs"])
@pytest.mark.parametrize("form", [grace.TF32, grace.BF16X3], ids=["tf32", "bf16x3"])
def test_grouped_step_equals_per_group_launches(form, pairs):
    # groups of very different sizes (N 16..80, k 0..3): several cell tiles for some groups,
    # ragged last tiles everywhere; the grouped and the per-group launches both on single CTAs or
    # both on CTA pairs (the same pairs of a group's cell tiles)
    specs, group, ic, dt = W.uneven_batch(900, seed=1107, n_range=(16, 80), orders=(0, 1, 2, 3))
    ctx = grace.Context(specs, 0, precisions=FORMS)
    b = ctx.batch(len(group), group)
    g0 = b.project(W.IC_EXP, ic)
    dtt = torch.as_tensor(dt, device=DEV)
    res = {}
    grace.set_cta_pairs(pairs)
    try:
        for grouped in (True, False):
            b.set_grouped(grouped)
            g = g0.clone()
            mass = torch.zeros(len(group), dtype=torch.float64, device=DEV)
            flags = torch.zeros(len(group), dtype=torch.uint8, device=DEV)
            b.step(g, dtt, 3, form, mass=mass, flags=flags)
            b.step(g, dtt, 2, form)
            res[grouped] = (g, mass, flags)
    finally:
        grace.set_cta_pairs(grace.CTA_PAIRS_NEVER)
    assert torch.equal(res[True][0], res[False][0])
    assert torch.equal(res[True][2], res[False][2])
    # the grouped K-c sums a cell's mass over 16 lanes; the per-group launch may use 32
    assert torch.allclose(res[True][1], res[False][1], rtol=1e-15, atol=0.0)
    assert b.device_error() == 0


@pytest.mark.parametrize("form", [grace.BF16X3], ids=["bf16x3"])
def test_grouped_step_matches_oracle(form):
    specs, group, ic, dt = W.uneven_batch(400, seed=1108, n_range=(16, 40), orders=(1, 2, 3))
    ctx = grace.Context(specs, 0, precisions=FORMS)
    b = ctx.batch(len(group), group)
    off = b.offsets()
    g = b.project(W.IC_EXP, ic)
    g0 = g.cpu().numpy()
    m0 = b.mass(g).cpu().numpy()
    mass = torch.zeros(len(group), dtype=torch.float64, device=DEV)
    b.step(g, torch.as_tensor(dt, device=DEV), 4, form, mass=mass)
    assert np.all(np.abs(mass.cpu().numpy() - m0) <= 1e-13 * np.abs(m0))
    gg = g.cpu().numpy()
    for gi, spec in enumerate(specs):
        idx = np.where(group == gi)[0]
        if idx.size == 0:
            continue
        o = oracle.Oracle(spec)
        go, mo, _ = o.step(np.stack(_split(g0, off, idx)), dt[idx], 4)
        h = np.diff(o.edges())
        d = np.abs(np.stack(_split(gg, off, idx)) - go).reshape(idx.size, spec.n_bins, -1).sum(axis=2)
        l1 = (h * d).sum(axis=1) / np.abs(mo)
        assert l1.max() <= 2e-5, (gi, l1.max())      # the BF16x3 trajectory bar (R15)
