"""Benchmark: DG coagulation RHS throughput in cell-steps/s on the batched additive-kernel workload.

Workload: 65,536 independent cells, K = x + y, N = 40 logarithmic bins on
[1e-6, 1e10], k = 2 (P = 120 coefficients per cell), conservative fluxes,
per-cell g0 = A x exp(-x/x0) with A ~ lognormal(0, 0.5), x0 ~ loguniform[1e-3, 1],
dt = 0.02 / (A x0^2).  One "step" is one SSP-RK3 step of the whole batch:
reconstruction (limiter), three flux contractions and three fused
flux-difference / RK-stage updates.

python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|tf32|bf16x3]
                [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference implementation
of this method available) on a bounded sample of the same workload.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DG RHS cell-steps/s (N=40,k=2) vs plain FP64 GPU; roofline frac; err vs FP64"
UNIT = "cell-steps/s"
FALLBACK_PEAKS = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}
# nominal dense rates of this part (TF32 relative to BF16; FP64 on CUDA cores)
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25
NOMINAL_FP64_TFLOPS = 1.25


def profiled_traffic(form_name):
    """DRAM bytes per launch of the contraction from the committed ncu summary of
    this form, or None when the kernel source changed since that capture."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", f"contract_tc_kernel_{form_name}_batched_additive_65536.md")
    src = os.path.join(ROOT, "paper_2607_13740_b300", "csrc", "grace_tc.cu")
    try:
        text = open(prof).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if f"sha256 prefix `{sha}`" not in text:
        return None
    for line in text.splitlines():
        if line.strip().startswith("traffic_bytes_per_launch:"):
            return int(line.split(":")[1])
    return None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as f:
                d = json.load(f)
            flat = {}

            def walk(x, prefix=""):
                if isinstance(x, dict):
                    for k, v in x.items():
                        walk(v, f"{prefix}{k}.")
                elif isinstance(x, (int, float)):
                    flat[prefix[:-1]] = float(x)
            walk(d)

            def pick(*names):
                for n in names:
                    for k, v in flat.items():
                        if k.split(".")[-1] == n:
                            return v
                return None
            peaks = {"hbm_gbs": pick("hbm_gbs"), "bf16_tflops": pick("bf16_tflops"),
                     "bf16_tflops_sustained": pick("bf16_tflops_sustained")}
            if all(v is not None for v in peaks.values()):
                peaks["source"] = "measured"
                return peaks
        except Exception:
            pass
    p = dict(FALLBACK_PEAKS)
    p["source"] = "fallback"
    return p


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(wl, n_steps_per_sample=1, target_s=12.0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload's cells."""
    import oracle
    o = oracle.Oracle(wl.spec)
    threads = oracle.max_threads()
    g0 = o.project(wl.ic_kind, wl.ic_params[:threads])
    t = time.perf_counter()
    o.step(g0, wl.dt[:threads], n_steps_per_sample, threads=threads)
    per = (time.perf_counter() - t)
    n = int(max(threads, min(4096, threads * max(1, target_s / max(per, 1e-6)))))
    n = min(n, wl.n_cells)
    g0 = o.project(wl.ic_kind, wl.ic_params[:n])
    t = time.perf_counter()
    o.step(g0, wl.dt[:n], n_steps_per_sample, threads=threads)
    el = time.perf_counter() - t
    return {"value": n * n_steps_per_sample / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {n} cells of the 65,536-cell batch x {n_steps_per_sample} SSP-RK3 step(s), "
                      f"FP64 C oracle with OpenMP, {el:.1f} s"}


def cpu_baseline_disk(spec, alpha, ic, n_cells=8):
    """The FP64 oracle, as it stands, on the first cells of the disk workload, one SSP-RK3 step
    each.  alpha is a parameter of the oracle's kernel, so every cell is its own oracle call (one
    core); the time step is the oracle's own (half its positivity bound at t = 0, untimed)."""
    import numpy as np
    import oracle
    from paper_2607_13740_b300 import workloads as W
    el = 0.0
    for c in range(n_cells):
        p = list(spec.coag_p)
        p[3] = float(alpha[c])
        o = oracle.Oracle(spec.replace(coag_p=tuple(p), frag_p=tuple(p), cell_alpha=0))
        g0 = o.project(W.IC_POWERLAW, ic[c:c + 1])
        L, _ = o.rhs(g0, threads=1)
        L0 = L.reshape(-1, spec.order_k + 1)[:, 0]
        m0 = g0.reshape(-1, spec.order_k + 1)[:, 0]
        neg = L0 < 0
        dt = 0.5 * float(np.min(m0[neg] / -L0[neg])) if neg.any() else 1.0
        t = time.perf_counter()
        o.step(g0, dt, 1, threads=1)
        el += time.perf_counter() - t
    return {"value": n_cells / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n_cells} cells of the disk batch (each with its own alpha) x 1 SSP-RK3 step, "
                      f"FP64 C oracle, one cell per call on one core, {el:.1f} s"}


def max_over_ranks(value, world, device):
    """The largest of every rank's value (timings: the job ends with its slowest rank); a
    collective only when world > 1 (gloo on CPU tensors, nccl on CUDA tensors)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, rank):
    """--impl reference: the oracle timed as it stands on bounded samples of the workload."""
    from paper_2607_13740_b300 import workloads as W
    if rank != 0:
        return
    import oracle
    wl = W.batched_additive(n_cells=args.cells or 65536)
    o = oracle.Oracle(wl.spec)
    threads = oracle.max_threads()
    n = max(threads, 2 * threads)
    g0 = o.project(wl.ic_kind, wl.ic_params[:n])
    times = []
    for s in range(args.warmup + args.steps):
        t = time.perf_counter()
        g0, _, _ = o.step(g0, wl.dt[:n], 1, threads=threads)
        if s >= args.warmup:
            times.append(time.perf_counter() - t)
    el = sum(times)
    value = n * len(times) / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "cells_per_step_sample": n, "n_bins": 40, "order_k": 2},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{n} of the 65,536 cells per step, FP64 C oracle with OpenMP"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_disk(args, emit=True):
    """Disk workload (per-cell alpha_turb, coagulation + fragmentation, N = 60): the node-space
    path in FP64 (a bounded 2,048 cells) or in a tensor-core form (262,144 cells by default:
    fixed pairs on tcgen05, partial entries in FP32); one JSON line like the headline's."""
    import torch
    from paper_2607_13740_b300 import grace, workloads as W
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    form = {"fp64": grace.FP64, "tf32": grace.TF32, "bf16x3": grace.BF16X3}[args.precision or "bf16x3"]
    fname = {grace.FP64: "fp64", grace.TF32: "tf32", grace.BF16X3: "bf16x3"}[form]
    n = args.cells or (2048 if form == grace.FP64 else 262144)
    steps = args.steps or (3 if form == grace.FP64 else 10)
    spec, alpha, ic = W.disk_batch(n_cells=n, order_k=args.order)
    t0 = time.time()
    ctx = grace.Context([spec], local, precisions=(grace.FP64, form) if form != grace.FP64 else (grace.FP64,))
    setup_s = time.time() - t0
    b = ctx.batch(n)
    b.cell_params(alpha)
    g0 = b.project(W.IC_POWERLAW, ic)
    # time step: half the positivity bound min_j g_j^0 / |L_j^0| at t = 0, held fixed
    L = b.rhs(g0, form).reshape(n, spec.n_bins, spec.order_k + 1)[:, :, 0]
    m = g0.reshape(n, spec.n_bins, spec.order_k + 1)[:, :, 0]
    ratio = torch.where(L < 0, m / (-L), torch.full_like(m, float("inf")))
    dt = 0.5 * ratio.amin(dim=1)
    dt = torch.where(torch.isfinite(dt), dt, torch.ones_like(dt))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    g = g0.clone()
    for _ in range(args.warmup):
        b.step(g, dt, 1, form)
    torch.cuda.synchronize()
    ctx.profile(True)
    for kk in range(3):
        ctx.profile_read(kk)
    sampler = ClockSampler(local)
    sampler.__enter__()
    evs = []
    for s_ in range(steps):
        flush.fill_(float(s_))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.step(g, dt, 1, form)
        e1.record()
        evs.append((e0, e1))
    torch.cuda.synchronize()
    sampler.__exit__(None, None, None)
    ms = sum(a.elapsed_time(c) for a, c in evs)
    c_ms, c_n = ctx.profile_read(0)
    u_ms, u_n = ctx.profile_read(1)
    x_ms, _ = ctx.profile_read(2)
    ctx.profile(False)
    avg = c_ms / max(1, c_n)
    peaks = load_peaks()
    if form == grace.FP64:
        macs, _ = ctx.stats(0, grace.FP64)          # multiply-adds of one RHS per cell (node-space path)
        achieved = 2.0 * macs * n / (avg / 1e3) / 1e12
        try:
            peak, psrc = 2.0 * grace.probe_rates(local)["fp64_fma_per_s"] / 1e12, "measured FP64 FMA rate x 2"
        except Exception:
            peak, psrc = NOMINAL_FP64_TFLOPS, "nominal FP64 rate"
        bound, kname = "alu", "node-space flux functionals (FP64)"
        alg = f"2 x {macs} multiply-adds per cell and RHS x {n} cells"
    else:
        tinfo = ctx.tile_info(0, form)
        passes = 3 if form == grace.BF16X3 else 1
        nz = tinfo["nnz_fold"]                      # non-zeros of the two fixed-pair tables
        achieved = 2.0 * nz * passes * n / (avg / 1e3) / 1e12
        if form == grace.TF32:
            peak = peaks["bf16_tflops_sustained"] * NOMINAL_TF32_OVER_BF16
            psrc = f"{peaks['source']} sustained bf16 x nominal tf32/bf16 ratio"
        else:
            peak, psrc = peaks["bf16_tflops_sustained"], f"{peaks['source']} sustained bf16"
        bound, kname = "tensor", "contract_tc_kernel (node-space tiles)"
        alg = f"2 x {nz} fixed-pair multiply-adds x {passes} MMA passes per cell and RHS x {n} cells"
        # the partial entries on the CUDA cores: 2 (k+1) + 2 multiply-adds per entry, cell and RHS
        # (the count behind grace_group_stats), against the measured FP32 FMA rate
        nnz_all, _ = ctx.stats(0, grace.FP64)
        per_entry = 2 * (spec.order_k + 1) + 2
        n_entries = (nnz_all - nz) // per_entry
        x_avg = x_ms / max(1, c_n)
        try:
            fp32_peak = 2.0 * grace.probe_rates(local)["fp32_fma_per_s"] / 1e12
            p32src = "measured FP32 FMA rate x 2"
        except Exception:
            fp32_peak, p32src = None, None
        ach32 = 2.0 * per_entry * n_entries * n / (x_avg / 1e3) / 1e12
        partial_roof = {"bound": "alu", "achieved": ach32, "peak": fp32_peak, "unit": "TFLOP/s",
                        "frac": ach32 / fp32_peak if fp32_peak else None,
                        "kernel": "nc_partial_f32_kernel + nc_pack_tc_kernel (timed together)",
                        "algorithmic": f"2 x {per_entry} multiply-adds x {n_entries} partial entries per cell "
                                       f"and RHS x {n} cells", "peak_source": p32src}
    m0 = b.mass(g0)
    drift = ((b.mass(g) - m0).abs() / m0.abs()).max().item()
    acc = None
    if form != grace.FP64:
        # accuracy of one RHS against the FP64 GPU path on the first 512 cells
        na = min(n, 512)
        bs = ctx.batch(na)
        bs.cell_params(alpha[:na])
        gs = g0.reshape(n, -1)[:na].reshape(-1).clone()
        L64 = bs.rhs(gs).reshape(na, -1)
        Lt = bs.rhs(gs, form).reshape(na, -1)
        acc = ((Lt - L64).abs().amax(dim=1) / L64.abs().amax(dim=1)).max().item()
    line = {
        "metric": "disk workload cell-steps/s (N=60, per-cell alpha, coag+frag)", "value": n * steps / (ms / 1e3),
        "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "tf32": "tf32", "bf16x3": "bf16x3"}[fname], "data": "synthetic",
        "config": {"workload": f"disk_{n}cells_N60_k{args.order}", "cells": n, "n_bins": 60, "order_k": args.order,
                   "form": fname, "alpha": "loguniform[1e-4, 1e-2] per cell", "ic": "MRN a^-3.5 over 1-10 um",
                   "dt": "0.5 x positivity bound at t=0", "precompute_s": setup_s,
                   "l2": "256 MB buffer written between timed steps (outside the timed events)"},
        "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel": kname, "algorithmic": alg,
                     "peak_source": psrc},
        "functionals_ms_avg": avg, "update_ms_avg": u_ms / max(1, u_n),
        "pack_and_partial_ms_per_stage": x_ms / max(1, c_n), "mass_drift": drift,
        "cpu_baseline": None if args.no_cpu_baseline else cpu_baseline_disk(spec, alpha, ic),
        "roofline_partial_entries": None if form == grace.FP64 else partial_roof,
        "max_rel_err_vs_fp64_rhs": acc, "finite": bool(torch.isfinite(g).all().item()),
        "clocks": sampler.summary(),
    }
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_adjoint(args, emit=True):
    """Adjoint workload: 4,096 cells of the disk physics (ballistic-turbulent kernels, fragmentation
    ramp, power-law fragments up to the larger collider plus the remnant) with one shared
    alpha_turb = 1e-3 on an N = 40, k = 2 grid of grain radii 1e-4 .. 1e2 cm; per-cell MRN initial
    states scaled by A ~ lognormal(0, 0.5); 200 SSP-RK3 steps with a checkpoint every 10; loss J =
    sum over cells of the final mass of grains above a radius (the exact polynomial integral of g
    above the grain mass of that radius; default 100 um: with alpha_turb = 1e-3 and v_frag = 1 m/s
    the fragmentation barrier holds the distribution near 30-90 um, and the mass above 1 mm stays
    ~1e-80 of the total, below the FP32 range of the tensor forms); gradients with respect to the
    initial coefficients, v_frag and the fragment exponent.
    Times grace_adjoint in the requested form (default bf16x3) next to the FP64 adjoint and the
    forward steps; one JSON line."""
    import numpy as np
    import torch
    from numpy.polynomial import legendre as npl
    from paper_2607_13740_b300 import grace, workloads as W
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    form = {"fp64": grace.FP64, "tf32": grace.TF32, "bf16x3": grace.BF16X3}[args.precision or "bf16x3"]
    fname = {grace.FP64: "fp64", grace.TF32: "tf32", grace.BF16X3: "bf16x3"}[form]
    n = args.cells or 4096
    steps, ckpt = args.steps or 200, 10
    spec = W.disk_spec(n_bins=40, order_k=2, cell_alpha=0, alpha=1e-3)
    _, _, ic1 = W.disk_batch(n_cells=1, n_bins=40, order_k=2)
    rng = np.random.default_rng(1005)
    ic = np.repeat(ic1, n, axis=0)
    ic[:, 0] *= rng.lognormal(0.0, 0.5, n)
    ctx = grace.Context([spec], local, precisions=(grace.FP64, form) if form != grace.FP64 else (grace.FP64,))
    # v_frag enters both ballistic kernels (coag_p[4], frag_p[4]); break_p[0] is the fragment exponent
    ctx.param_grad_setup([4, 12, 16])
    b = ctx.batch(n)
    g0 = b.project(W.IC_POWERLAW, ic)
    # time step: half the positivity bound at t = 0 per cell (as the disk workload), held fixed
    L = b.rhs(g0).reshape(n, 40, 3)[:, :, 0]
    m = g0.reshape(n, 40, 3)[:, :, 0]
    ratio = torch.where(L < 0, m / (-L), torch.full_like(m, float("inf")))
    dt = (0.5 * ratio.amin(dim=1)).contiguous()
    dt = torch.where(torch.isfinite(dt), dt, torch.ones_like(dt))
    # lambda_T = dJ/dg_T: J = int_{x_cut}^{x_max} g dx, x_cut the mass of a 0.1 cm grain
    edges = spec.x_min * (spec.x_max / spec.x_min) ** (np.arange(41) / 40)
    edges[0], edges[-1] = spec.x_min, spec.x_max
    x_cut = W.grain_mass(args.loss_radius)
    lam = np.zeros((40, 3))
    for j in range(40):
        a_, b_ = edges[j], edges[j + 1]
        if b_ <= x_cut:
            continue
        xi0 = -1.0 if a_ >= x_cut else 2.0 * (x_cut - 0.5 * (a_ + b_)) / (b_ - a_)
        for i in range(3):
            c = np.zeros(i + 1)
            c[i] = 1.0
            anti = npl.legint(c)
            lam[j, i] = 0.5 * (b_ - a_) * (npl.legval(1.0, anti) - npl.legval(xi0, anti))
    lamT = torch.as_tensor(np.tile(lam.reshape(-1), (n, 1)), device=dev).contiguous()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    sampler = ClockSampler(local)
    sampler.__enter__()
    ms_adj, (lam0, dth) = timed(lambda: b.adjoint(g0, dt, steps, lamT, ckpt, param_grads=True, precision=form))
    sampler.__exit__(None, None, None)
    ms_fwd, _ = timed(lambda: b.step(g0.clone(), dt, steps, form))
    res = {"adjoint_ms": ms_adj, "forward_ms": ms_fwd, "adjoint_over_forward": ms_adj / ms_fwd}
    if form != grace.FP64 and not args.skip_fp64_compare:
        # like-for-like comparison with the FP64 adjoint: the first 512 cells, 20 steps, both forms
        ns, cs = min(n, 512), min(steps, 20)
        bs = ctx.batch(ns)
        g0s = g0.reshape(n, -1)[:ns].contiguous().clone()
        lamTs = lamT.reshape(n, -1)[:ns].contiguous().clone()
        dts = dt[:ns].contiguous().clone()
        ms_s, (lam_s, dth_s) = timed(lambda: bs.adjoint(g0s, dts, cs, lamTs, ckpt, param_grads=True, precision=form))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        lam64, dth64 = bs.adjoint(g0s, dts, cs, lamTs, ckpt, param_grads=True, precision=grace.FP64)
        e1.record()
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        lam_s, lam64 = lam_s.reshape(ns, -1), lam64.reshape(ns, -1)
        res["comparison"] = {
            "cells": ns, "steps": cs, "form_ms": ms_s, "fp64_ms": ms64, "speedup_vs_fp64_adjoint": ms64 / ms_s,
            "lambda0_max_rel_err_vs_fp64": ((lam_s - lam64).abs().amax(dim=1) /
                                            lam64.abs().amax(dim=1).clamp_min(1e-300)).max().item(),
            "dtheta_max_rel_err_vs_fp64": ((dth_s - dth64).abs().amax(dim=0) /
                                           dth64.abs().amax(dim=0).clamp_min(1e-300)).max().item(),
            "dtheta_sum_fp64": dth64.sum(dim=0).tolist(), "dtheta_sum_form": dth_s.sum(dim=0).tolist()}
    line = {
        "metric": "adjoint cell-steps/s (4,096 cells, N=40, k=2, disk physics one alpha, 200 steps, ckpt 10)",
        "value": n * steps / (ms_adj / 1e3), "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": 1,
        "ms_per_step": ms_adj / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "tf32": "tf32", "bf16x3": "bf16x3"}[fname], "data": "synthetic",
        "config": {"workload": f"adjoint_{n}cells_N40_k2_disk", "cells": n, "form": fname, "checkpoint_every": ckpt,
                   "physics": "ballistic-turbulent kernels, alpha_turb = 1e-3 shared, ramp over 0.8..1.2 v_frag, "
                              "power law -11/6 up to the larger collider + remnant",
                   "loss": f"final mass of grains above radius {args.loss_radius} cm (exact polynomial integral)",
                   "params": ["v_frag (coag_p[4] + frag_p[4])", "fragment exponent"],
                   "ic": "MRN g ~ x^(-5/6) over 1..10 um, scaled by A ~ lognormal(0, 0.5)",
                   "dt": "0.5 x positivity bound at t = 0 per cell"},
        "finite": bool(torch.isfinite(lam0).all().item() and torch.isfinite(dth).all().item()),
        "J": float((lamT * b.step(g0.clone(), dt, steps, grace.FP64 if form == grace.FP64 else form)).sum()),
        "dJ_dtheta": {"v_frag": float(dth[:, 0].sum() + dth[:, 1].sum()), "fragment_exponent": float(dth[:, 2].sum())},
        "clocks": sampler.summary(), **res,
    }
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_uneven(args, emit=True):
    """Uneven batch: cells of many groups (N ~ U{16..80}, k ~ U{0..3}, constant or additive
    kernel, per-cell rate scale) stepped together in the bf16x3 form: per-group launch sequences
    and the grouped step (one multi-group contraction and one K-c launch per stage), each direct
    and replayed from a CUDA graph.  One JSON line (value: grouped, graph)."""
    import torch
    from paper_2607_13740_b300 import grace, workloads as W
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    n = args.cells or 100000
    steps = args.steps or 3
    specs, group, ic, dt_np = W.uneven_batch(n_cells=n)
    t0 = time.time()
    ctx = grace.Context(specs, local, precisions=(grace.FP64, grace.BF16X3))
    setup_s = time.time() - t0
    b = ctx.batch(n, group)
    g0 = b.project(W.IC_EXP, ic)
    dt = torch.as_tensor(dt_np, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    side = torch.cuda.Stream(device=dev)     # graph capture needs a non-default stream
    passes = 3
    alg = 2.0 * passes * sum(ctx.tile_info(gi, grace.BF16X3)["nnz_fold"] * int((group == gi).sum())
                             for gi in range(len(specs)))
    variants = [v for v in (("per_group", False, False), ("per_group_graph", False, True),
                            ("grouped", True, False), ("grouped_graph", True, True))
                if args.variants is None or v[0] in args.variants.split(",")]
    for name, grouped, graph in variants:
        b.set_grouped(grouped)
        b.set_graph(graph)
        g = g0.clone()
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            for _ in range(args.warmup):
                b.step(g, dt, 1, grace.BF16X3)
            prof = grouped and not graph
            if prof:
                ctx.profile(True)
                ctx.profile_read(0)
                ctx.profile_read(1)
            evs = []
            sampler = ClockSampler(local) if name == "grouped_graph" else None
            if sampler:
                sampler.__enter__()
            for s_ in range(steps):
                flush.fill_(float(s_))
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(side)
                b.step(g, dt, 1, grace.BF16X3)
                e1.record(side)
                evs.append((e0, e1))
        torch.cuda.synchronize()
        if sampler:
            sampler.__exit__(None, None, None)
        ms = sum(a.elapsed_time(c) for a, c in evs)
        res[name] = {"ms_per_step": ms / steps, "cell_steps_per_s": n * steps / (ms / 1e3),
                     "finite": bool(torch.isfinite(g).all().item())}
        if prof:
            c_ms, c_n = ctx.profile_read(0)
            u_ms, u_n = ctx.profile_read(1)
            ctx.profile(False)
            res[name]["contract_ms_avg"] = c_ms / max(1, c_n)
            res[name]["update_ms_avg"] = u_ms / max(1, u_n)
        if sampler:
            res[name]["clocks"] = sampler.summary()
    b.set_graph(False)
    peaks = load_peaks()
    cavg = res["grouped"]["contract_ms_avg"] if "grouped" in res else float("nan")
    achieved = alg / (cavg / 1e3) / 1e12
    tiles = [ctx.tile_info(i, grace.BF16X3) for i in range(len(specs))]
    counts = [int((group == gi).sum()) for gi in range(len(specs))]
    b_stream = float(sum(t["b_bytes"] * ((c + 127) // 128) for t, c in zip(tiles, counts)))
    # A operand (BF16 hi + lo of the padded coefficients) read, FP32 functionals written, per cell
    af_bytes = float(sum(c * (4 * ((sp.n_coef + 63) // 64 * 64) + 4 * (sp.n_bins - 1 + sp.n_bins * sp.order_k))
                         for sp, c in zip(specs, counts)))
    best = res.get("grouped_graph") or res.get("grouped") or next(iter(res.values()))
    line = {
        "metric": "uneven-batch cell-steps/s (bf16x3, one multi-group launch per stage, CUDA graph)",
        "value": best["cell_steps_per_s"],
        "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": best["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic",
        "config": {"workload": f"uneven_{n}cells_{len(specs)}groups", "cells": n, "groups": len(specs),
                   "N": "U{16..80}", "k": "U{0..3}", "kernels": "constant / additive", "precompute_s": setup_s,
                   "l2": "256 MB buffer written between timed steps (outside the timed events)"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_tflops"],
                     "unit": "TFLOP/s", "frac": achieved / peaks["bf16_tflops"],
                     "frac_sustained": achieved / peaks["bf16_tflops_sustained"], "traffic": None,
                     "kernel": "contract_tc_kernel (multi-group mode)",
                     "algorithmic": "2 x (non-zeros of the folded tables of the cell's group) x 3 passes, summed over cells",
                     "peak_source": f"{peaks['source']} burst bf16 (a sub-ms launch)",
                     # every work item streams its group's B image; with one or two tiles per group
                     # the images cannot stay in L2, so the launch also has an HBM view
                     "hbm": {"b_image_bytes_per_launch": b_stream,
                             "a_and_f_bytes_per_launch": af_bytes,
                             "achieved_gbs": (b_stream + af_bytes) / (cavg / 1e3) / 1e9,
                             "peak_gbs": peaks["hbm_gbs"],
                             "frac": (b_stream + af_bytes) / (cavg / 1e3) / 1e9 / peaks["hbm_gbs"]}},
        "clocks": best.get("clocks"), "variants": res,
        "tiles": {"mma_per_tile_min": min(t["mma_per_tile"] for t in tiles),
                  "mma_per_tile_max": max(t["mma_per_tile"] for t in tiles),
                  "folded_groups": sum(t["folded"] for t in tiles)},
    }
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_eoc(args):
    """Paper-scale convergence study (Sec. 4.2, eq. eoc) on the GPU in FP64: constant kernel K = 1,
    non-conservative fluxes on [1e-3, 1e15], f(x, 0) = exp(-x) (g0 = x exp(-x)), to tau = 3e12 against
    eq. (fcoagsolution), N in {10, 20, 40, 100, 200} and k in {0..4}; time step dt = c (2 + tau), a
    fixed fraction c of the collision time of the self-similar solution.  Errors e_c (16 Gauss points
    per bin) and e_d (geometric bin centres) of Sec. 4.1, the relative error of M_1, and the EOC
    ln(e_N / e_N') / ln(N' / N) between successive N.  One JSON line."""
    import numpy as np
    import torch
    from numpy.polynomial import legendre as npl
    from paper_2607_13740_b300 import grace, workloads as W
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    tau_end = float(args.tau or 3e12)
    c = float(args.eoc_c)
    Ns = [int(x) for x in (args.eoc_n or "10,20,40,100,200").split(",")]
    ks = [int(x) for x in (args.eoc_k or "0,1,2,3,4").split(",")]
    s16, w16 = npl.leggauss(16)

    def exact(x, t):
        return x * 4.0 / (2.0 + t) ** 2 * np.exp(-2.0 * x / (2.0 + t))

    def errors(coef, e, k, t):
        coef = coef.reshape(len(e) - 1, k + 1)
        h, xc = np.diff(e), 0.5 * (e[1:] + e[:-1])
        x = xc[:, None] + 0.5 * h[:, None] * s16[None, :]
        gh = np.stack([npl.legval(s16, coef[j]) for j in range(len(e) - 1)])
        ec = float((0.5 * h * (w16[None, :] * np.abs(gh - exact(x, t))).sum(axis=1)).sum())
        xg = np.sqrt(e[1:] * e[:-1])
        gd = np.array([npl.legval(2.0 * (xg[j] - xc[j]) / h[j], coef[j]) for j in range(len(e) - 1)])
        ed = float((h * np.abs(gd - exact(xg, t))).sum())
        return ec, ed

    res, t0_all = {}, time.time()
    for k in ks:
        for N in Ns:
            spec = W.constant_kernel_spec(N, k, W.FLUX_NONCONSERVATIVE, 1e-3, 1e15)
            ctx = grace.Context([spec], local)
            b = ctx.batch(1)
            g = b.project(W.IC_EXP, [[1.0, 1.0, 0.0, 0.0]])
            dt = torch.zeros(1, dtype=torch.float64, device=dev)
            t, n_steps = 0.0, 0
            torch.cuda.synchronize()
            tw = time.time()
            while t < tau_end * (1.0 - 1e-15):
                step = min(c * (2.0 + t), tau_end - t)
                dt.fill_(step)
                b.step(g, dt, 1, grace.FP64)
                t += step
                n_steps += 1
            torch.cuda.synchronize()
            wall = time.time() - tw
            e = spec.x_min * (spec.x_max / spec.x_min) ** (np.arange(N + 1) / N)
            e[0], e[-1] = spec.x_min, spec.x_max
            coef = g.cpu().numpy().reshape(-1)
            ec, ed = errors(coef, e, k, t)
            m1 = float((np.diff(e) * coef.reshape(N, k + 1)[:, 0]).sum())
            res[(k, N)] = {"e_c": ec, "e_d": ed, "mass_rel_err": abs(m1 - 1.0), "steps": n_steps, "gpu_wall_s": wall,
                           "finite": bool(np.isfinite(coef).all())}
    eoc = {}
    for k in ks:
        eoc[k] = []
        for N1, N2 in zip(Ns[:-1], Ns[1:]):
            a, b_ = res[(k, N1)]["e_c"], res[(k, N2)]["e_c"]
            eoc[k].append(math.log(a / b_) / math.log(N2 / N1) if a > 0 and b_ > 0 else None)
    line = {
        "metric": "EOC of the constant-kernel test (Sec. 4.2) at tau = 3e12, FP64 on the GPU", "unit": "order",
        "value": {str(k): eoc[k][-1] for k in ks}, "n_gpus": 1, "data": "synthetic (analytic test problem)",
        "dtype": "f64", "higher_is_better": True,
        "config": {"workload": "constant_kernel_eoc", "x_range": [1e-3, 1e15], "flux": "non-conservative",
                   "ic": "f(x,0) = exp(-x)", "tau_end": tau_end, "dt": f"{c} (2 + tau)", "N": Ns, "k": ks},
        "eoc_per_k": {str(k): eoc[k] for k in ks},
        "errors": {f"k{k}_N{N}": v for (k, N), v in res.items()},
        "paper": "EOC = k + 1 for N = 10..200, k = 0..4; e_c < 1% at k = 4 with N = 40",
        "wall_s": time.time() - t0_all,
    }
    print(json.dumps(line), flush=True)


def run_toy(args):
    """The coupled aggregation-breakage toy model of Sec. 4.5 on the GPU in FP64: Maxwellian
    relative velocities (dv_rms = 0.5, v_b = 0.1, v_f = 1), power-law fragments with index -1.83
    plus a remnant (eqs. break, mfrag), non-conservative fluxes on [1e-6, 1e3], f(x, 0) = exp(-x).
    Runs the paper's N = 20 solutions (k = 0..3) and its reference resolution N = 300, k = 4 with
    dt = 0.05, and reports at each output time the low-mass slope d ln g / d ln x (least squares
    over the bin means of the bins centred in [1e-5, 1e-2]), the L1 distance of each N = 20
    solution from the reference, the mass M_1 and the status bits.  One JSON line."""
    import numpy as np
    import torch
    from numpy.polynomial import legendre as npl
    from paper_2607_13740_b300 import grace, workloads as W
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    taus = [float(x) for x in (args.toy_tau or "1,10,100").split(",")]
    dt_val = float(args.toy_dt)
    runs = [(20, k) for k in range(4)] + [(int(args.toy_ref_n), 4)]
    s16, w16 = npl.leggauss(16)
    out, states, t_all = {}, {}, time.time()
    for N, k in runs:
        spec = W.coupled_toy_spec(N, k)
        ctx = grace.Context([spec], local)
        b = ctx.batch(1)
        g = b.project(W.IC_EXP, [[1.0, 1.0, 0.0, 0.0]])
        dt = torch.full((1,), dt_val, dtype=torch.float64, device=dev)
        flags = torch.zeros(1, dtype=torch.uint8, device=dev)
        e = spec.x_min * (spec.x_max / spec.x_min) ** (np.arange(N + 1) / N)
        e[0], e[-1] = spec.x_min, spec.x_max
        h, xc = np.diff(e), np.sqrt(e[1:] * e[:-1])
        sel = (xc >= 1e-5) & (xc <= 1e-2)
        t, rec = 0.0, {}
        torch.cuda.synchronize()
        tw = time.time()
        for tau in taus:
            n = int(round((tau - t) / dt_val))
            b.step(g, dt, n, grace.FP64, flags=flags)
            t += n * dt_val
            coef = g.cpu().numpy().reshape(N, k + 1)
            means = coef[:, 0]
            ok = sel & (means > 0)
            slope = float(np.polyfit(np.log(xc[ok]), np.log(means[ok]), 1)[0]) if ok.sum() >= 2 else None
            # local slopes between neighbouring bin means over the fit range (is it one power law?)
            loc = np.diff(np.log(np.where(means > 0, means, np.nan))) / np.diff(np.log(xc))
            mid = np.sqrt(xc[1:] * xc[:-1])
            in_fit = (mid >= 1e-5) & (mid <= 1e-2) & np.isfinite(loc)
            rec[f"{tau:g}"] = {"slope": slope, "mass": float((h * means).sum()), "flags": int(flags.item()),
                               "finite": bool(np.isfinite(coef).all()),
                               "local_slope_range": [float(loc[in_fit].min()), float(loc[in_fit].max())]
                               if in_fit.any() else None}
            if in_fit.any():
                # the flattest stretch of log g over the fit range: the largest local slope, and the
                # masses where the local slope stays within 0.01 of it (where a power law reads best)
                i_pl = int(np.argmax(np.where(in_fit, loc, -np.inf)))
                near = in_fit & (loc >= loc[i_pl] - 0.01)
                rec[f"{tau:g}"]["plateau"] = {"slope": float(loc[i_pl]), "x": float(mid[i_pl]),
                                              "x_range": [float(mid[near].min()), float(mid[near].max())]}
            if k == 4:
                # the reference's slope profile over the whole grid: (x between bins, local slope)
                rec[f"{tau:g}"]["local_slopes"] = [[float(a), float(b)] for a, b in zip(mid, loc) if np.isfinite(b)]
            states[(N, k, tau)] = (e, coef)
        torch.cuda.synchronize()
        out[f"N{N}_k{k}"] = {"tau": rec, "steps": int(round(t / dt_val)), "gpu_wall_s": time.time() - tw}

    def evaluate(e, coef, x):
        j = np.clip(np.searchsorted(e, x, side="right") - 1, 0, len(e) - 2)
        xi = 2.0 * (x - 0.5 * (e[j] + e[j + 1])) / (e[j + 1] - e[j])
        return np.array([npl.legval(xi[i], coef[j[i]]) for i in range(len(x))])

    ref_n = int(args.toy_ref_n)
    for tau in taus:
        er, cr = states[(ref_n, 4, tau)]
        hr, xr = np.diff(er), 0.5 * (er[1:] + er[:-1])
        x = (xr[:, None] + 0.5 * hr[:, None] * s16[None, :]).ravel()
        w = (0.5 * hr[:, None] * w16[None, :]).ravel()
        gref = evaluate(er, cr, x)
        for k in range(4):
            e20, c20 = states[(20, k, tau)]
            d = float((w * np.abs(evaluate(e20, c20, x) - gref)).sum() / (w * np.abs(gref)).sum())
            out[f"N20_k{k}"]["tau"][f"{tau:g}"]["l1_vs_reference"] = d
    line = {
        "metric": "coupled aggregation-breakage toy model (Sec. 4.5): low-mass slope and distance from the "
                  "N = 300, k = 4 reference, FP64 on the GPU", "unit": "d ln g / d ln x",
        "value": (out[f"N{ref_n}_k4"]["tau"][f"{taus[-1]:g}"].get("plateau") or {}).get("slope"), "n_gpus": 1,
        "data": "synthetic (the paper's test problem)", "dtype": "f64", "higher_is_better": None,
        "config": {"workload": "coupled_toy", "x_range": [1e-6, 1e3], "flux": "non-conservative",
                   "ic": "f(x,0) = exp(-x)", "dt": dt_val, "tau": taus, "runs": [f"N{N}_k{k}" for N, k in runs],
                   "slope_fit": "bin means of the bins centred in [1e-5, 1e-2]",
                   "value": "the reference's plateau slope at the last output time: the largest local slope "
                            "d ln g / d ln x between neighbouring bin means in [1e-5, 1e-2]"},
        "paper": "g ~ x^-0.748 at the low-mass end (Birnstiel et al. 2011 scaling with nu = 2/3, alpha = -1.83)",
        "runs": out, "wall_s": time.time() - t_all,
    }
    print(json.dumps(line), flush=True)


def run_species(args, emit=True):
    """Species of mixed grains (Sec. 5.3): the batched additive workload's 65,536 cells split into
    S = 2 species (a tracer holding the two smallest bins, and the rest), stepped with
    grace_step_species in a tensor form (default bf16x3): one tcgen05 pass over T per stage for
    both species.  CUDA events around one call of K steps; one JSON line (cell-steps/s counts
    cells, each carrying S distributions)."""
    import torch
    from paper_2607_13740_b300 import grace, workloads as W
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    form = {"fp64": grace.FP64, "tf32": grace.TF32, "bf16x3": grace.BF16X3}[args.precision or "bf16x3"]
    wl = W.batched_additive(n_cells=args.cells or 65536)
    n, steps = wl.n_cells, args.steps or 10
    ctx = grace.Context([wl.spec], local, precisions=(grace.FP64, form) if form != grace.FP64 else (grace.FP64,))
    b = ctx.batch(n)
    g = b.project(wl.ic_kind, wl.ic_params)
    tracer = torch.zeros_like(g).reshape(n, wl.spec.n_bins, -1)
    tracer[:, :2, :] = g.reshape(n, wl.spec.n_bins, -1)[:, :2, :]
    tracer = tracer.reshape(n, -1)
    gs0 = torch.stack([tracer, g - tracer]).contiguous()
    dt = torch.as_tensor(wl.dt, device=dev)
    gs = gs0.clone()
    for _ in range(args.warmup):
        b.step_species(gs, dt, 1, form)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    gs.copy_(gs0)
    flush.fill_(1.0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record()
        b.step_species(gs, dt, steps, form)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    fname = {grace.FP64: "fp64", grace.TF32: "tf32", grace.BF16X3: "bf16x3"}[form]
    line = {
        "metric": "species cell-steps/s (S = 2 distributions per cell, N=40, k=2)", "value": n * steps / (ms / 1e3),
        "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "dtype": fname, "data": "synthetic",
        "config": {"workload": f"species2_{n}cells_N40_k2", "cells": n, "species": 2,
                   "split": "tracer = the two smallest bins, the rest", "timing": f"one grace_step_species call of {steps} steps"},
        "finite": bool(torch.isfinite(gs).all().item()), "clocks": clk.summary(),
    }
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_mv(args, emit=True):
    """Two-dimensional (mass, volume) DG of Sec. 5.3: 16,384 independent cells of 12 x 12 bins over four
    decades in each coordinate, k = 1 (576 coefficients per cell), the mixed five-term kernel, the
    contraction in FP64 (or FP32 with --mv-arith fp32; the state stays FP64); one grace_mv_step call
    of `steps` SSP-RK3 steps timed with CUDA events (the state and the step workspace, about 300 MB,
    exceed the 126 MB L2)."""
    import torch
    from paper_2607_13740_b300 import grace, workloads as W
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    n = args.cells or 16384
    steps = args.steps or 5
    spec, g0_np, dt_np = W.mv_batch(n_cells=n)
    t0 = time.time()
    fp32 = getattr(args, "mv_arith", "fp64") == "fp32"
    mv = grace.MV(spec, local, fp32=fp32)
    setup_s = time.time() - t0
    g0 = torch.as_tensor(g0_np, device=dev)
    dt = torch.as_tensor(dt_np, device=dev)
    g = g0.clone()
    for _ in range(max(1, args.warmup)):
        mv.step(g, dt, 1)
    torch.cuda.synchronize()
    g = g0.clone()
    sampler = ClockSampler(local)
    sampler.__enter__()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    mv.step(g, dt, steps)
    e1.record()
    torch.cuda.synchronize()
    sampler.__exit__(None, None, None)
    ms = e0.elapsed_time(e1)
    # the contraction alone, for its roofline: three RHS launches
    L = torch.empty_like(g0)
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    r0.record()
    for _ in range(3):
        mv.rhs(g0, out=L)
    r1.record()
    torch.cuda.synchronize()
    rhs_ms = r0.elapsed_time(r1) / 3
    # multiply-adds of one RHS and cell as executed: per term the loss (a bilinear scalar and the
    # cell-local operator) and the gain (per target row a: H = Xg[a] G, W = G^T H, then <Vg[b], W>,
    # each over the source bins that can land in the target)
    K1 = spec.order_k + 1
    Px, Pv = spec.n_x * K1, spec.n_v * K1
    P = Px * Pv
    vsum = sum(((b // K1 + 1) * K1) ** 2 for b in range(Pv))
    gain = sum(((a // K1 + 1) * K1) ** 2 * Pv + Pv * Pv * ((a // K1 + 1) * K1) + vsum for a in range(Px))
    macs = len(spec.terms) * (P + P * K1 * K1 + gain)
    achieved = 2.0 * macs * n / (rhs_ms / 1e3) / 1e12
    key, name = ("fp32_fma_per_s", "FP32") if fp32 else ("fp64_fma_per_s", "FP64")
    try:
        peak, psrc = 2.0 * grace.probe_rates(local)[key] / 1e12, f"measured {name} FMA rate x 2"
    except Exception:
        peak, psrc = (None, "FP32 rate not measured") if fp32 else (NOMINAL_FP64_TFLOPS, "nominal FP64 rate")
    # mass sum_{j,m} h_j h_m g^{00}: no merger leaves the grid in these steps, so it changes only by
    # the quadrature difference of the gain and loss rules
    ex = spec.x_min * (spec.x_max / spec.x_min) ** (np.arange(spec.n_x + 1) / spec.n_x)
    ev = spec.v_min * (spec.v_max / spec.v_min) ** (np.arange(spec.n_v + 1) / spec.n_v)
    w = (np.diff(ex)[:, None] * np.diff(ev)[None, :]).reshape(-1)
    def mass(t):
        return (t.cpu().numpy().reshape(n, spec.n_x, K1, spec.n_v, K1)[:, :, 0, :, 0].reshape(n, -1) * w).sum(axis=1)
    m0, m1 = mass(g0), mass(g)
    line = {"metric": f"2-D (mass, volume) DG cell-steps/s (Sec. 5.3; 12 x 12 bins, k = 1, 5-term kernel, {name})",
            "value": n * steps / (ms / 1e3), "unit": "cell-steps/s", "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if fp32 else "f64", "data": "synthetic",
            "config": {"workload": f"mv_{n}cells_{spec.n_x}x{spec.n_v}_k{spec.order_k}" + ("_fp32" if fp32 else ""),
                       "cells": n, "contraction_arithmetic": name.lower(),
                       "n_x": spec.n_x, "n_v": spec.n_v, "order_k": spec.order_k, "quad_q": spec.quad_q,
                       "coef_per_cell": P, "kernel_terms": len(spec.terms),
                       "l2": "state + step workspace about 300 MB, larger than the 126 MB L2",
                       "timing": "one grace_mv_step call, CUDA events on the launching stream"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak if peak else None, "traffic": None,
                         "kernel": ("mv_rhs_f32_kernel" if fp32 else "mv_rhs_kernel") + f" ({name} contraction of the factor forms)",
                         "algorithmic": f"2 x {macs} multiply-adds per cell and RHS x {n} cells", "peak_source": psrc},
            "rhs_ms": rhs_ms, "setup_s": setup_s,
            "mass_drift": float(np.abs(m1 - m0).max() / np.abs(m0).max()),
            "clocks": sampler.summary()}
    if emit:
        print(json.dumps(line))
    return line


def run_legs(args):
    """Short runs of the other configurations after the headline (N = 1 only), so that their
    figures come from the same command: the uneven batch (grouped step, graph-replayed, 3 steps),
    the adjoint leg (bf16x3, no FP64 comparison), the disk workload (65,536 cells, k = 2,
    bf16x3, 3 steps), species (bf16x3, 10 steps) and the two-dimensional (mass, volume) DG (16,384
    cells, 3 steps, FP64 and FP32 contractions).  Each leg's own JSON line is summarised; a failing leg records its error and
    never affects the headline."""
    import copy
    import torch
    out = {}
    base = copy.copy(args)
    base.steps, base.cells, base.precision, base.variants, base.forms = None, None, None, None, None
    plans = [
        ("uneven", run_uneven, {"steps": 3, "variants": "grouped_graph,grouped"}),
        ("adjoint", run_adjoint, {"skip_fp64_compare": True}),
        ("disk", run_disk, {"cells": 65536, "steps": 3, "order": 2, "precision": "bf16x3"}),
        ("species", run_species, {"steps": 10, "precision": "bf16x3"}),
        ("mv", run_mv, {"steps": 3, "mv_arith": "fp64"}),
        ("mv_fp32", run_mv, {"steps": 3, "mv_arith": "fp32"}),
    ]
    for name, fn, over in plans:
        a = copy.copy(base)
        for k, v in over.items():
            setattr(a, k, v)
        t0 = time.time()
        try:
            ln = fn(a, emit=False)
            keep = {k: ln.get(k) for k in ("metric", "value", "unit", "ms_per_step", "dtype", "roofline", "clocks")}
            keep["workload"] = (ln.get("config") or {}).get("workload")
            if name == "adjoint":
                keep["dJ_dtheta"] = ln.get("dJ_dtheta")
                keep["adjoint_over_forward"] = ln.get("adjoint_over_forward")
            out[name] = keep
        except Exception as exc:          # a leg never takes the headline down
            out[name] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
        out[name]["wall_s"] = time.time() - t0
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, choices=["fp64", "tf32", "bf16x3"])
    ap.add_argument("--cells", type=int, default=None,
                    help="cells of the workload (default: 65,536 additive, 262,144 disk tensor forms / 2,048 FP64, "
                         "4,096 adjoint, 100,000 uneven)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--skip-fp64-compare", action="store_true", help="adjoint workload: no FP64 comparison run")
    ap.add_argument("--forms", default=None,
                    help="comma-separated subset of fp64,tf32,bf16x3 to time (default: all built)")
    ap.add_argument("--tau", type=float, default=None, help="eoc workload: end time (default 3e12)")
    ap.add_argument("--loss-radius", type=float, default=0.01,
                    help="adjoint workload: the loss is the final mass of grains above this radius (cm)")
    ap.add_argument("--eoc-c", type=float, default=0.02, help="eoc workload: dt = c (2 + tau)")
    ap.add_argument("--eoc-n", default=None, help="eoc workload: comma-separated bin counts")
    ap.add_argument("--eoc-k", default=None, help="eoc workload: comma-separated degrees")
    ap.add_argument("--toy-tau", default=None, help="toy workload: comma-separated output times (default 1,10,100)")
    ap.add_argument("--toy-dt", type=float, default=0.05, help="toy workload: time step")
    ap.add_argument("--toy-ref-n", type=int, default=300, help="toy workload: bins of the k = 4 reference")
    ap.add_argument("--workload", default="additive",
                    choices=["additive", "disk", "uneven", "adjoint", "eoc", "toy", "species", "mv"],
                    help="additive: the batched additive-kernel headline; disk: coagulation + fragmentation "
                         "with a per-cell turbulence strength (node-space path); uneven: many groups in one batch; "
                         "adjoint: checkpointed adjoint of 200 steps with parameter gradients")
    ap.add_argument("--order", type=int, default=2, help="disk workload: Legendre degree k (1..3)")
    ap.add_argument("--mv-arith", default="fp64", choices=["fp64", "fp32"],
                    help="mv workload: arithmetic of the contraction (the state stays FP64)")
    ap.add_argument("--no-legs", action="store_true",
                    help="additive workload: skip the short uneven / adjoint / disk legs reported under 'legs'")
    ap.add_argument("--variants", default=None,
                    help="uneven workload: comma-separated subset of per_group,per_group_graph,grouped,grouped_graph")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.workload == "disk":
        run_disk(args)
        return
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "uneven":
        run_uneven(args)
        return
    if args.workload == "toy":
        return run_toy(args)
    if args.workload == "mv":
        run_mv(args)
        return
    if args.workload == "species":
        run_species(args)
        return
    if args.workload == "eoc":
        run_eoc(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if args.steps is None:
            args.steps = 3
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    from paper_2607_13740_b300 import grace, workloads as W

    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    # weak scaling: each rank steps its own share of a global batch of world x the per-rank cells
    n_rank = args.cells or 65536
    wl = W.shard(W.batched_additive(n_cells=n_rank * world), rank, world) if world > 1 else \
        W.batched_additive(n_cells=n_rank)
    n = wl.n_cells
    candidates = [grace.FP64, grace.TF32, grace.BF16X3]
    ctx = None
    for forms in (candidates, [grace.FP64]):
        try:
            ctx = grace.Context([wl.spec], local, precisions=forms)
            break
        except grace.GraceError:
            ctx = None
    forms = list(ctx.precisions)
    if args.forms:
        want = [grace.PRECISIONS[f.strip()] for f in args.forms.split(",") if f.strip()]
        forms = [f for f in forms if f in want]
    head = grace.PRECISIONS[args.precision] if args.precision else forms[-1]
    if head not in forms:
        raise SystemExit(f"precision {args.precision} was not precomputed by the library")
    if args.steps is None:
        args.steps = 3 if head == grace.FP64 else 100
    b = ctx.batch(n)
    g0 = b.project(wl.ic_kind, wl.ic_params)
    dt = torch.as_tensor(wl.dt, device=dev)
    nnz, _ = ctx.stats(0, grace.FP64)
    peaks = load_peaks()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    names = {grace.FP64: "fp64", grace.TF32: "tf32", grace.BF16X3: "bf16x3"}

    def timed(form, steps, warmup, clocks=False, one_call=False):
        """K steps timed with CUDA events on the launching stream: one grace_step call of K steps
        (one_call; the configured workload is one call of 100 steps) or K calls of one step each
        (every call pays the step-start conversion and the FP64 output of its last stage)."""
        g = g0.clone()
        for _ in range(warmup):
            b.step(g, dt, 1, form)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ctx.profile(True)
        ctx.profile_read(0)
        ctx.profile_read(1)
        evs = []
        sampler = ClockSampler(local) if clocks else None
        if sampler:
            sampler.__enter__()
        torch.cuda.synchronize()
        for s in range(1 if one_call else steps):
            flush.fill_(float(s))            # evict L2 before every timed call (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            b.step(g, dt, steps if one_call else 1, form)
            e1.record()
            evs.append((e0, e1))
        torch.cuda.synchronize()
        if sampler:
            sampler.__exit__(None, None, None)
        ms = sum(a.elapsed_time(c) for a, c in evs)
        c_ms, c_n = ctx.profile_read(0)
        u_ms, u_n = ctx.profile_read(1)
        ctx.profile(False)
        ms_max = max_over_ranks(ms, world, dev)
        if world > 1:
            dist.barrier()
        return {"ms": ms_max, "contract_ms": c_ms, "contract_launches": c_n, "update_ms": u_ms,
                "update_launches": u_n, "g": g, "clocks": sampler.summary() if sampler else None,
                "calls": 1 if one_call else steps}

    # accuracy of each form against the FP64 GPU path over the same steps
    err_steps = 3
    ref = g0.clone()
    b.step(ref, dt, err_steps, grace.FP64)
    m0 = b.mass(g0)
    edges = torch.as_tensor(np.array([wl.spec.x_min * (wl.spec.x_max / wl.spec.x_min) ** (j / 40)
                                      for j in range(41)]), device=dev)
    h = (edges[1:] - edges[:-1])

    # roofline denominators: the tensor-core forms are timed as sub-ms launches inside sub-ms steps,
    # so their peak is the burst rate: the measured cuBLAS bf16 burst for BF16x3 (MEASURED_PEAKS.json),
    # and this project's own tcgen05 kind::tf32 probe (M = 128, N = 256) for TF32; the probe's
    # single-product bf16 rate is reported beside it
    mma_peaks = {}
    for pf, key in ((grace.TF32, "tf32"), (grace.BF16X3, "bf16")):
        try:
            mma_peaks[key] = grace.probe_mma(pf, 256, local) / 1e12
        except Exception as exc:
            mma_peaks[key + "_error"] = str(exc)[:120]
    survey_nnz = 410000          # the scope table's estimate of the non-zeros of T for N = 40, k = 2

    def roofline(form, avg_ms, tinfo):
        """The contraction's achieved rate per launch on three algorithmic bases and its fraction
        of the form's peak; the primary basis is the exact non-zero count of T (the scope table's
        per-cell figure, counted by the precompute instead of estimated)."""
        passes = 3 if form == grace.BF16X3 else 1
        sec = avg_ms / 1e3
        bases = {"T_nonzeros_exact": nnz, "survey_estimate": survey_nnz}
        if tinfo:
            bases["folded_nonzeros"] = tinfo["nnz_fold"]
        ach = {k: 2.0 * v * n * passes / sec / 1e12 for k, v in bases.items()}
        if form == grace.FP64:
            try:
                fma64 = grace.probe_rates(local)["fp64_fma_per_s"]   # measured on this GPU
                peak, psrc = 2.0 * fma64 / 1e12, "measured FP64 FMA rate (grace_probe_rates) x 2 flop"
            except Exception:
                peak, psrc = NOMINAL_FP64_TFLOPS, "nominal FP64 rate of the part (1.25 TFLOP/s)"
            return {"bound": "alu", "achieved": ach["T_nonzeros_exact"], "peak": peak, "unit": "TFLOP/s",
                    "frac": ach["T_nonzeros_exact"] / peak, "peak_source": psrc,
                    "bases": {k: {"nonzeros_per_cell": bases[k], "achieved": a, "frac": a / peak}
                              for k, a in ach.items()}}
        if form == grace.TF32 and "tf32" in mma_peaks:
            peak, psust = mma_peaks["tf32"], None
            psrc = "measured tcgen05 kind::tf32 rate (grace_probe_mma, M = 128, N = 256), burst"
        elif form == grace.TF32:
            peak = peaks["bf16_tflops"] * NOMINAL_TF32_OVER_BF16
            psust, psrc = None, f"{peaks['source']} burst bf16 x nominal tf32/bf16 ratio"
        else:
            peak, psust = peaks["bf16_tflops"], peaks["bf16_tflops_sustained"]
            psrc = f"{peaks['source']} burst bf16 (cuBLAS)"
        out = {"bound": "tensor", "achieved": ach["T_nonzeros_exact"], "peak": peak, "unit": "TFLOP/s",
               "frac": ach["T_nonzeros_exact"] / peak, "frac_burst": ach["T_nonzeros_exact"] / peak,
               "peak_source": psrc,
               "bases": {k: {"nonzeros_per_cell": bases[k], "achieved": a, "frac_burst": a / peak}
                         for k, a in ach.items()}}
        if psust:
            out["frac_sustained"] = ach["T_nonzeros_exact"] / psust
            out["peak_sustained"] = psust
            for k, a in ach.items():
                out["bases"][k]["frac_sustained"] = a / psust
        return out

    forms_out = {}
    for form in forms:
        is_head = form == head
        steps = args.steps if is_head else min(args.steps, 3 if form == grace.FP64 else 20)
        # the headline form: one grace_step call of K steps (the configured workload at K = 100),
        # next to K calls of one step; the other forms: one-step calls
        r = timed(form, steps, args.warmup if is_head else 1, clocks=is_head, one_call=is_head)
        r1 = timed(form, min(steps, 20), 1) if is_head else r
        cell_steps = n * world * steps / (r["ms"] / 1e3)
        tinfo = ctx.tile_info(0, form) if form != grace.FP64 else None
        avg = r["contract_ms"] / max(1, r["contract_launches"])
        g = g0.clone()
        b.step(g, dt, err_steps, form)
        d = (g - ref).abs().reshape(n, 40, 3)
        l1 = ((h[None, :] * d.sum(dim=2)).sum(dim=1) / m0.abs()).max().item()
        mx = (d.amax(dim=(1, 2)) / ref.reshape(n, 40, 3).abs().amax(dim=(1, 2))).max().item()
        mass = b.mass(g)
        drift = ((mass - m0).abs() / m0.abs()).max().item()
        forms_out[names[form]] = {
            "cell_steps_per_s": cell_steps, "ms_per_step": r["ms"] / steps, "steps": steps,
            "timing": f"one grace_step call of {steps} steps" if is_head else f"{steps} one-step calls",
            "contract_ms_avg": avg, "contract_launches": r["contract_launches"], "tiles": tinfo,
            "update_ms_avg": r["update_ms"] / max(1, r["update_launches"]),
            "update_launches": r["update_launches"],
            "roofline": roofline(form, avg, tinfo),
            "l1_err_vs_fp64_over_M1": l1, "max_rel_err_vs_fp64": mx, "mass_drift": drift,
            "err_steps": err_steps, "_r": r}
        if is_head:
            s1 = min(steps, 20)
            forms_out[names[form]]["one_step_calls"] = {
                "cell_steps_per_s": n * world * s1 / (r1["ms"] / 1e3), "ms_per_step": r1["ms"] / s1, "steps": s1,
                "contract_ms_avg": r1["contract_ms"] / max(1, r1["contract_launches"]),
                "update_ms_avg": r1["update_ms"] / max(1, r1["update_launches"])}

    hd = forms_out[names[head]]
    r = hd.pop("_r")
    for f in forms_out.values():
        f.pop("_r", None)
    if "fp64" in forms_out:
        fp64_rate = forms_out["fp64"]["cell_steps_per_s"]
        for f in forms_out.values():
            f["speedup_vs_fp64_gpu"] = f["cell_steps_per_s"] / fp64_rate

    # end to end through the public API: pinned host state in, one step, state out
    e2e = None
    if args.no_e2e:
        e2e = {"value": None, "unit": UNIT, "skipped": "--no-e2e"}
    try:
        if args.no_e2e:
            raise StopIteration
        # every step goes through grace_step_host (the C ABI on host buffers): the state and
        # the time steps are uploaded from page-locked host memory, stepped, and the new state
        # downloaded, inside the call; successive calls are independent batches, so the library's
        # double-buffered staging overlaps the upload of step i+1 and the download of step i-1
        # with the compute of step i
        host_in = g0.cpu().pin_memory()
        host_dt = dt.cpu().pin_memory()
        outs = [torch.empty_like(host_in).pin_memory() for _ in range(2)]
        e2e_steps = max(3, min(args.steps, 20))

        def host_steps(n_steps):
            for i in range(n_steps):
                b.step_host(host_in, host_dt, 1, head, out=outs[i % 2])
            b.wait_host()

        host_steps(2)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        host_steps(e2e_steps)
        torch.cuda.synchronize()
        ems = (time.perf_counter() - t0) * 1e3
        if not torch.isfinite(outs[(e2e_steps - 1) % 2]).all():
            raise RuntimeError("non-finite state after the host-buffer steps")
        ems_max = max_over_ranks(ems, world, dev)
        nbytes = host_in.numel() * 8
        e2e = {"value": n * world * e2e_steps / (ems_max / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": nbytes + host_dt.numel() * 8, "d2h_bytes_per_step": nbytes,
               "steps": e2e_steps, "api": "grace_step_host (C ABI, host buffers), host wall clock",
               "pipelining": "the library's double-buffered staging overlaps the upload of step i+1 "
                             "and the download of step i-1 with the compute of step i "
                             "(independent batches, page-locked host buffers, two copy streams)"}
    except StopIteration:
        pass
    except Exception as exc:  # pinned memory may be unavailable
        e2e = {"value": None, "unit": UNIT, "error": str(exc)[:200]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl)

    # kernels of the timed region: the contractions and stage updates counted by the launch
    # timers, plus the one step-start limiter of each call
    gpu_launches = r["contract_launches"] + r["update_launches"] + r["calls"]
    line = {
        "metric": METRIC, "value": hd["cell_steps_per_s"], "unit": UNIT, "n_gpus": world,
        "steps": hd["steps"], "warmup": args.warmup, "ms_per_step": hd["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {grace.FP64: "f64", grace.TF32: "tf32", grace.BF16X3: "bf16x3"}[head],
        "data": "synthetic",
        "config": {"workload": wl.name.split("_shard")[0], "cells_per_gpu": n, "global_batch": n * world,
                   "n_bins": 40, "order_k": 2,
                   "coef_per_cell": wl.spec.n_coef, "kernel": "additive K=x+y", "flux": "conservative",
                   "x_range": [wl.spec.x_min, wl.spec.x_max], "precision": names[head],
                   "l2": "256 MB buffer written before every timed call (outside the timed events); inside "
                         "a multi-step call the working set (state, three compact stage states, functionals, "
                         "A operand: about 250 MB) exceeds the 126 MB L2",
                   "timing": f"one grace_step call of {hd['steps']} steps, CUDA events on the launching stream; "
                             "forms.<precision>.one_step_calls has K calls of one step",
                   "parallelism": f"dp{world} (independent cells, no collective on the data path)"},
        "roofline": {**{k: v for k, v in hd["roofline"].items() if k != "bases"},
                     "traffic": profiled_traffic(names[head]) if head != grace.FP64 else None,
                     "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum per launch, committed ncu "
                                       "summary (null when the kernel changed since)",
                     "kernel": "flux contraction",
                     "algorithmic": f"2 x {nnz} non-zeros of T per cell and RHS (exact count of the scope "
                                    f"table's per-cell figure) x {n} cells"
                                    + (" x 3 bf16 passes" if head == grace.BF16X3 else ""),
                     "bases": hd["roofline"]["bases"],
                     "tf32_peak_measured": mma_peaks.get("tf32"), "bf16_single_product_peak_measured":
                         mma_peaks.get("bf16")},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": r["clocks"],
        "forms": forms_out,
        "peaks": peaks,
    }
    if rank == 0 and world == 1 and not args.no_legs:
        line["legs"] = run_legs(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
