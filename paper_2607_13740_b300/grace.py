"""Thin ctypes binding of the C ABI in include/grace.h (argument marshalling only).

Device buffers are torch tensors on the context's CUDA device; every compute
call runs on torch's current stream.  There is no CPU fallback: if the
library or a CUDA device is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgrace.so")

FP64, TF32, BF16X3 = 0, 1, 2
PRECISIONS = {"fp64": FP64, "tf32": TF32, "bf16x3": BF16X3}
FLAG_NEGATIVE_MEAN, FLAG_LIMITED, FLAG_NONFINITE, FLAG_CFL, FLAG_MASS_DRIFT = 1, 2, 4, 8, 16
WARN_CELLS = 100

_lib = None
_VP = ctypes.c_void_p


class GraceError(RuntimeError):
    pass


class GroupDesc(ctypes.Structure):
    _fields_ = [
        ("n_bins", ctypes.c_int), ("order_k", ctypes.c_int), ("quad_q", ctypes.c_int),
        ("flux_mode", ctypes.c_int), ("coag_kind", ctypes.c_int), ("frag_kind", ctypes.c_int),
        ("break_kind", ctypes.c_int), ("cutoff_mode", ctypes.c_int), ("limiter", ctypes.c_int),
        ("mfrag_mode", ctypes.c_int),
        ("x_min", ctypes.c_double), ("x_max", ctypes.c_double),
        ("coag_p", ctypes.c_double * 8), ("frag_p", ctypes.c_double * 8),
        ("break_p", ctypes.c_double * 8),
        ("cell_alpha", ctypes.c_int), ("reserved_", ctypes.c_int),
        ("edges", ctypes.POINTER(ctypes.c_double)),
    ]


def exported_symbols():
    return ["grace_version", "grace_status_string", "grace_last_error", "grace_setup",
            "grace_set_stream", "grace_precompute", "grace_group_info", "grace_bind_batch",
            "grace_batch_offsets", "grace_project", "grace_rhs", "grace_step", "grace_mass",
            "grace_limit", "grace_profile_enable", "grace_profile_read", "grace_group_stats",
            "grace_batch_error", "grace_rhs_jvp", "grace_rhs_vjp", "grace_param_grad_setup",
            "grace_adjoint", "grace_probe_rates", "grace_batch_set_graph", "grace_batch_set_grouped", "grace_batch_destroy",
            "grace_destroy", "grace_tile_info", "grace_batch_cell_params", "grace_rhs_noalloc",
            "grace_step_host", "grace_step_host_wait", "grace_flags_check",
            "grace_test_arm_wait_timeout", "grace_set_cta_pairs", "grace_set_tc_a_in_tmem", "grace_probe_mma", "grace_substep", "grace_rhs_species",
            "grace_step_species", "grace_rosenbrock_step", "grace_mv_setup", "grace_mv_set_stream", "grace_mv_rhs",
            "grace_mv_step", "grace_mv_destroy"]


def load(path: str | None = None):
    """Loads libgrace.so (built in-tree by paper_2607_13740_b300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise GraceError(f"CUDA library not built: {path} (run paper_2607_13740_b300.build)")
    L = ctypes.CDLL(path)
    S = ctypes.c_int
    L.grace_version.restype = ctypes.c_int
    L.grace_status_string.argtypes = [S]
    L.grace_status_string.restype = ctypes.c_char_p
    L.grace_last_error.restype = ctypes.c_char_p
    L.grace_setup.argtypes = [ctypes.POINTER(_VP), S, ctypes.POINTER(GroupDesc), S]
    L.grace_set_stream.argtypes = [_VP, _VP]
    L.grace_precompute.argtypes = [_VP, ctypes.c_uint]
    L.grace_group_info.argtypes = [_VP, S, ctypes.POINTER(S), ctypes.POINTER(S)]
    L.grace_bind_batch.argtypes = [_VP, S, _VP, ctypes.POINTER(_VP)]
    L.grace_batch_offsets.argtypes = [_VP, ctypes.POINTER(ctypes.c_longlong)]
    L.grace_project.argtypes = [_VP, S, _VP, _VP]
    L.grace_rhs.argtypes = [_VP, _VP, _VP, S]
    L.grace_step.argtypes = [_VP, _VP, _VP, S, S, _VP, _VP]
    L.grace_mass.argtypes = [_VP, _VP, _VP]
    L.grace_limit.argtypes = [_VP, _VP, _VP]
    L.grace_profile_enable.argtypes = [_VP, S]
    L.grace_profile_read.argtypes = [_VP, S, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
    L.grace_group_stats.argtypes = [_VP, S, S, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    L.grace_batch_error.argtypes = [_VP, ctypes.POINTER(S)]
    L.grace_tile_info.argtypes = [_VP, S, S, ctypes.POINTER(ctypes.c_longlong)]
    L.grace_batch_cell_params.argtypes = [_VP, _VP]
    L.grace_rhs_jvp.argtypes = [_VP, _VP, _VP, _VP, S]
    L.grace_rhs_vjp.argtypes = [_VP, _VP, _VP, _VP, S]
    L.grace_param_grad_setup.argtypes = [_VP, S, S, _VP, ctypes.c_double]
    L.grace_adjoint.argtypes = [_VP, _VP, _VP, S, S, _VP, _VP, _VP, S]
    L.grace_probe_rates.argtypes = [S, ctypes.POINTER(ctypes.c_double)]
    L.grace_probe_mma.argtypes = [S, S, S, ctypes.POINTER(ctypes.c_double)]
    L.grace_rhs_species.argtypes = [_VP, S, _VP, _VP, S]
    L.grace_rosenbrock_step.argtypes = [_VP, _VP, _VP, S, S, S, ctypes.c_double, ctypes.POINTER(S)]
    L.grace_step_species.argtypes = [_VP, S, _VP, _VP, S, S, _VP, _VP]
    L.grace_substep.argtypes = [_VP, _VP, _VP, ctypes.c_double, S, S, _VP, _VP, ctypes.POINTER(S)]
    L.grace_batch_set_graph.argtypes = [_VP, S]
    L.grace_batch_set_grouped.argtypes = [_VP, S]
    L.grace_step_host.argtypes = [_VP, _VP, _VP, _VP, S, S, _VP, _VP]
    L.grace_step_host_wait.argtypes = [_VP]
    L.grace_flags_check.argtypes = [_VP, _VP, ctypes.POINTER(ctypes.c_uint)]
    L.grace_test_arm_wait_timeout.argtypes = [ctypes.c_longlong]
    L.grace_set_cta_pairs.argtypes = [ctypes.c_int]
    L.grace_set_tc_a_in_tmem.argtypes = [ctypes.c_int]
    L.grace_mv_setup.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    L.grace_mv_set_stream.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.grace_mv_rhs.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    L.grace_mv_step.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    L.grace_mv_destroy.argtypes = [ctypes.c_void_p]
    L.grace_mv_destroy.restype = None
    L.grace_batch_destroy.argtypes = [_VP]
    L.grace_destroy.argtypes = [_VP]
    for name in exported_symbols():
        if not hasattr(L, name):
            raise GraceError(f"{path} does not export {name}")
    _lib = L
    return L


def _check(status: int, what: str):
    if status != 0:
        L = load()
        msg = L.grace_status_string(status).decode()
        detail = L.grace_last_error().decode()
        raise GraceError(f"{what}: {msg} ({detail})")


def group_desc(spec: W.GroupSpec) -> GroupDesc:
    d = GroupDesc()
    for f in ("n_bins", "order_k", "quad_q", "flux_mode", "coag_kind", "frag_kind", "break_kind",
              "cutoff_mode", "limiter", "mfrag_mode", "x_min", "x_max", "cell_alpha"):
        setattr(d, f, getattr(spec, f))
    for name in ("coag_p", "frag_p", "break_p"):
        arr = getattr(d, name)
        for i, v in enumerate(getattr(spec, name)):
            arr[i] = v
    if spec.edges is not None:
        buf = (ctypes.c_double * len(spec.edges))(*spec.edges)
        d.edges = ctypes.cast(buf, ctypes.POINTER(ctypes.c_double))
        d._edges_buf = buf          # alive as long as the descriptor
    return d


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream_handle():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def arm_wait_timeout(wait_cycles: int):
    """One-shot failure-detection check: the next tensor-core contraction launch issues no
    operand copies and its bounded waits give up after wait_cycles (grace_test_arm_wait_timeout)."""
    _check(load().grace_test_arm_wait_timeout(int(wait_cycles)), "grace_test_arm_wait_timeout")


CTA_PAIRS_NEVER, CTA_PAIRS_ALWAYS, CTA_PAIRS_MULTI = 0, 1, 2


def set_cta_pairs(mode: int):
    """Process-wide: where forward contractions in the tensor forms run on CTA pairs
    (cta_group::2): CTA_PAIRS_NEVER (the default), CTA_PAIRS_ALWAYS or CTA_PAIRS_MULTI
    (multi-group launches only) (grace_set_cta_pairs)."""
    _check(load().grace_set_cta_pairs(int(mode)), "grace_set_cta_pairs")


def set_tc_a_in_tmem(enable: bool):
    """Process-wide: single-group forward contractions in the tensor forms keep the A tile in
    tensor memory or in shared memory (the default) (grace_set_tc_a_in_tmem)."""
    _check(load().grace_set_tc_a_in_tmem(1 if enable else 0), "grace_set_tc_a_in_tmem")


def probe_rates(device: int = 0):
    """Measured CUDA-core rates on this device: FP64 FMA/s, FP32 FMA/s, FP64->FP32 conversions/s."""
    out = (ctypes.c_double * 3)()
    _check(load().grace_probe_rates(int(device), out), "grace_probe_rates")
    return {"fp64_fma_per_s": out[0], "fp32_fma_per_s": out[1], "f64_to_f32_cvt_per_s": out[2]}


def probe_mma(precision: int, n: int = 256, device: int = 0) -> float:
    """Measured dense tcgen05.mma rate (FLOP/s) with M = 128 and the given N: kind::tf32 for
    TF32, kind::f16 with bf16 operands for BF16X3 (one product per instruction)."""
    out = ctypes.c_double()
    _check(load().grace_probe_mma(int(device), int(precision), int(n), ctypes.byref(out)), "grace_probe_mma")
    return out.value


class MVDesc(ctypes.Structure):
    """grace_mv_desc: the two-dimensional (mass, volume) grid, degree, rule and kernel terms."""
    _fields_ = [
        ("n_x", ctypes.c_int), ("n_v", ctypes.c_int), ("order_k", ctypes.c_int), ("quad_q", ctypes.c_int),
        ("x_min", ctypes.c_double), ("x_max", ctypes.c_double), ("v_min", ctypes.c_double),
        ("v_max", ctypes.c_double), ("n_terms", ctypes.c_int),
        ("coef", ctypes.c_double * 8), ("ax", ctypes.c_double * 8), ("bx", ctypes.c_double * 8),
        ("av", ctypes.c_double * 8), ("bv", ctypes.c_double * 8), ("arithmetic", ctypes.c_int),
    ]


def mv_desc(spec, fp32: bool = False) -> MVDesc:
    d = MVDesc()
    d.n_x, d.n_v, d.order_k, d.quad_q = spec.n_x, spec.n_v, spec.order_k, spec.quad_q
    d.x_min, d.x_max, d.v_min, d.v_max = spec.x_min, spec.x_max, spec.v_min, spec.v_max
    d.n_terms = len(spec.terms)
    for t, (c, ax, bx, av, bv) in enumerate(spec.terms):
        d.coef[t], d.ax[t], d.bx[t], d.av[t], d.bv[t] = c, ax, bx, av, bv
    d.arithmetic = 1 if fp32 else 0
    return d


class MV:
    """Two-dimensional (mass, volume) DG of Sec. 5.3 (grace_mv_*): g and L are float64 CUDA tensors
    [n_cells, n_coef] in the layout ((j (k+1) + p) n_v + m)(k+1) + q; fp32 selects the FP32
    contraction (the state stays FP64)."""

    def __init__(self, spec, device: int = 0, fp32: bool = False):
        self.spec = spec
        self.device = device
        self._h = ctypes.c_void_p()
        d = mv_desc(spec, fp32)
        _check(load().grace_mv_setup(ctypes.byref(self._h), ctypes.byref(d), int(device)), "grace_mv_setup")

    def _stream(self):
        _check(load().grace_mv_set_stream(self._h, _stream_handle()), "grace_mv_set_stream")

    def _state(self, g):
        import torch
        if not (g.is_cuda and g.dtype == torch.float64 and g.is_contiguous() and g.dim() == 2
                and g.shape[1] == self.spec.n_coef):
            raise GraceError("g must be a contiguous float64 CUDA tensor [n_cells, n_coef]")

    def rhs(self, g, out=None):
        import torch
        self._state(g)
        L = out if out is not None else torch.empty_like(g)
        self._stream()
        _check(load().grace_mv_rhs(self._h, int(g.shape[0]), _ptr(g), _ptr(L)), "grace_mv_rhs")
        return L

    def step(self, g, dt, n_steps: int):
        """n_steps SSP-RK3 steps in place; dt a float64 CUDA tensor [n_cells]."""
        self._state(g)
        self._stream()
        _check(load().grace_mv_step(self._h, int(g.shape[0]), _ptr(g), _ptr(dt), int(n_steps)), "grace_mv_step")
        return g

    def close(self):
        if self._h:
            load().grace_mv_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """Setup + FP64 precompute (and tensor-core tiles for the requested precisions)."""

    def __init__(self, specs, device: int = 0, precisions=(FP64,)):
        import torch
        if not torch.cuda.is_available():
            raise GraceError("no CUDA device: the GRACE-DG library has no CPU path")
        L = load()
        self.specs = list(specs) if isinstance(specs, (list, tuple)) else [specs]
        self.device = device
        descs = [group_desc(s) for s in self.specs]    # hold their edge buffers through the setup call
        arr = (GroupDesc * len(descs))(*descs)
        h = _VP()
        torch.cuda.set_device(device)
        _check(L.grace_setup(ctypes.byref(h), len(self.specs), arr, device), "grace_setup")
        del descs
        self._h = h
        self.set_stream()
        mask = 0
        for p in precisions:
            mask |= 1 << int(p)
        _check(L.grace_precompute(h, mask), "grace_precompute")
        self.precisions = tuple(int(p) for p in precisions)

    def set_stream(self):
        _check(load().grace_set_stream(self._h, _stream_handle()), "grace_set_stream")

    def group_info(self, group: int = 0):
        P, R = ctypes.c_int(), ctypes.c_int()
        _check(load().grace_group_info(self._h, group, ctypes.byref(P), ctypes.byref(R)), "grace_group_info")
        return P.value, R.value

    def profile(self, enable: bool = True):
        _check(load().grace_profile_enable(self._h, 1 if enable else 0), "grace_profile_enable")

    def profile_read(self, kernel: int):
        """(total device ms, launches) of kernel 0 (contraction) or 1 (flux update) since the last read."""
        ms, n = ctypes.c_double(), ctypes.c_longlong()
        _check(load().grace_profile_read(self._h, kernel, ctypes.byref(ms), ctypes.byref(n)), "grace_profile_read")
        return ms.value, n.value

    def stats(self, group: int = 0, precision: int = FP64):
        """(non-zeros of the coefficient tensors, executed tile MACs) per cell and RHS."""
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        _check(load().grace_group_stats(self._h, group, precision, ctypes.byref(a), ctypes.byref(b)),
               "grace_group_stats")
        return a.value, b.value

    def tile_info(self, group: int = 0, precision: int = TF32) -> dict:
        """The tensor-core tile plan of a group (grace_tile_info)."""
        a = (ctypes.c_longlong * 8)()
        _check(load().grace_tile_info(self._h, group, precision, a), "grace_tile_info")
        keys = ("n_tiles", "mma_per_tile", "mac_per_cell", "b_bytes", "pred_clk_per_tile", "max_n", "nnz_fold",
                "folded")
        return dict(zip(keys, list(a)))

    def param_grad_setup(self, param_ids, group: int = 0, rel_step: float = 0.0):
        """Enables dJ/dtheta in Batch.adjoint for kernel parameters given by id:
        0..7 coag_p[i], 8..15 frag_p[i-8], 16..23 break_p[i-16]."""
        ids = np.ascontiguousarray(param_ids, dtype=np.int32)
        _check(load().grace_param_grad_setup(self._h, group, len(ids), ids.ctypes.data_as(ctypes.c_void_p),
                                             float(rel_step)), "grace_param_grad_setup")
        self.param_ids = tuple(int(i) for i in ids)

    def batch(self, n_cells: int, cell_group=None) -> "Batch":
        return Batch(self, n_cells, cell_group)

    def close(self):
        if getattr(self, "_h", None):
            load().grace_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    def __init__(self, ctx: Context, n_cells: int, cell_group=None):
        self.ctx = ctx
        self.n_cells = n_cells
        self._host_pending = []
        h = _VP()
        cg = None
        if cell_group is not None:
            cg_arr = np.ascontiguousarray(cell_group, dtype=np.int32)
            cg = cg_arr.ctypes.data_as(ctypes.c_void_p)
        _check(load().grace_bind_batch(ctx._h, n_cells, cg, ctypes.byref(h)), "grace_bind_batch")
        self._h = h
        self.group0 = int(np.asarray(cell_group).reshape(-1)[0]) if cell_group is not None else 0
        self.P, self.R = ctx.group_info(self.group0)
        self.mixed = cell_group is not None and len(set(np.asarray(cell_group).tolist())) > 1
        self.total = int(self.offsets()[-1])

    def offsets(self):
        out = (ctypes.c_longlong * (self.n_cells + 1))()
        _check(load().grace_batch_offsets(self._h, out), "grace_batch_offsets")
        return np.frombuffer(out, dtype=np.int64).copy()

    def _check_state(self, g):
        import torch
        if not (g.is_cuda and g.dtype == torch.float64 and g.is_contiguous()):
            raise GraceError("coefficient arrays must be contiguous float64 CUDA tensors")
        if g.numel() != self.total:
            raise GraceError(f"expected {self.total} coefficients, got {g.numel()}")

    def project(self, ic_kind: int, ic_params):
        import torch
        ic = torch.as_tensor(np.ascontiguousarray(ic_params, dtype=np.float64)).reshape(self.n_cells, 4)
        ic = ic.to(f"cuda:{self.ctx.device}")
        g = torch.empty(self.total, dtype=torch.float64, device=ic.device)
        if not self.mixed:
            g = g.view(self.n_cells, self.P)
        self.ctx.set_stream()
        _check(load().grace_project(self._h, int(ic_kind), _ptr(ic), _ptr(g)), "grace_project")
        return g

    def rhs(self, g, precision: int = FP64, out=None):
        import torch
        self._check_state(g)
        L = out if out is not None else torch.empty_like(g)
        self.ctx.set_stream()
        _check(load().grace_rhs(self._h, _ptr(g), _ptr(L), int(precision)), "grace_rhs")
        return L

    def step(self, g, dt, n_steps: int, precision: int = FP64, mass=None, flags=None):
        """In place on g; dt is a float64 CUDA tensor [n_cells]."""
        self._check_state(g)
        self.ctx.set_stream()
        _check(load().grace_step(self._h, _ptr(g), _ptr(dt), int(n_steps), int(precision),
                                 _ptr(mass), _ptr(flags)), "grace_step")
        return g

    def rhs_species(self, gs, precision: int = FP64):
        """Species of mixed grains: gs [S, n_cells, P] float64 CUDA tensor of partial mass densities;
        returns L_s = L[g_s; sum_s g_s] in the same layout (grace_rhs_species)."""
        import torch
        if not (gs.is_cuda and gs.dtype == torch.float64 and gs.is_contiguous() and gs.dim() == 3):
            raise GraceError("gs must be a contiguous float64 CUDA tensor [S, n_cells, P]")
        out = torch.empty_like(gs)
        self.ctx.set_stream()
        _check(load().grace_rhs_species(self._h, gs.shape[0], _ptr(gs), _ptr(out), int(precision)),
               "grace_rhs_species")
        return out

    def step_species(self, gs, dt, n_steps: int, precision: int = FP64, mass=None, flags=None):
        """n_steps SSP-RK3 steps of the species, in place on gs [S, n_cells, P] (grace_step_species)."""
        import torch
        if not (gs.is_cuda and gs.dtype == torch.float64 and gs.is_contiguous() and gs.dim() == 3):
            raise GraceError("gs must be a contiguous float64 CUDA tensor [S, n_cells, P]")
        self.ctx.set_stream()
        _check(load().grace_step_species(self._h, gs.shape[0], _ptr(gs), _ptr(dt), int(n_steps), int(precision),
                                         _ptr(mass), _ptr(flags)), "grace_step_species")
        return gs

    def rosenbrock_step(self, g, dt, precision: int = FP64, krylov_dim: int = 30, max_restarts: int = 4,
                        rtol: float = 1e-10) -> int:
        """One linearly implicit Euler step per cell, in place on g: (I - dt J) k = dt L[g], g += k,
        solved by restarted GMRES on the JVPs (grace_rosenbrock_step).  Returns the Krylov
        iterations taken."""
        self._check_state(g)
        self.ctx.set_stream()
        it = ctypes.c_int(0)
        _check(load().grace_rosenbrock_step(self._h, _ptr(g), _ptr(dt), int(precision), int(krylov_dim),
                                            int(max_restarts), float(rtol), ctypes.byref(it)), "grace_rosenbrock_step")
        return it.value

    def substep(self, g, dt_hydro, cfl: float = 0.5, max_substeps: int = 1000, precision: int = FP64, mass=None,
                flags=None) -> int:
        """Advances every cell by its own dt_hydro (float64 CUDA tensor [n_cells]) in sub-steps sized by
        the eq. (dt) bound (grace_substep); in place on g; returns the number of sub-steps taken."""
        self._check_state(g)
        nsub = ctypes.c_int()
        self.ctx.set_stream()
        _check(load().grace_substep(self._h, _ptr(g), _ptr(dt_hydro), float(cfl), int(max_substeps), int(precision),
                                    _ptr(mass), _ptr(flags), ctypes.byref(nsub)), "grace_substep")
        return nsub.value

    def _check_host(self, t, numel, dtype, what):
        import torch
        if t.is_cuda or t.dtype != dtype or not t.is_contiguous() or t.numel() != numel:
            raise GraceError(f"{what} must be a contiguous {dtype} host tensor of {numel} elements")

    def step_host(self, g, dt, n_steps: int, precision: int = FP64, out=None, mass=None, flags=None):
        """grace_step on host tensors (float64 g [total] and dt [n_cells]; out, mass, flags host
        tensors or None; out defaults to g).  Returns once the work is enqueued: read the
        outputs after wait_host().  Page-locked tensors let successive calls overlap."""
        import torch
        self._check_host(g, self.total, torch.float64, "g")
        self._check_host(dt, self.n_cells, torch.float64, "dt")
        out = g if out is None else out
        self._check_host(out, self.total, torch.float64, "out")
        if mass is not None:
            self._check_host(mass, self.n_cells, torch.float64, "mass")
        if flags is not None:
            self._check_host(flags, self.n_cells, torch.uint8, "flags")
        self.ctx.set_stream()
        _check(load().grace_step_host(self._h, _ptr(g), _ptr(out), _ptr(dt), int(n_steps), int(precision),
                                      _ptr(mass), _ptr(flags)), "grace_step_host")
        self._host_pending.append((g, dt, out, mass, flags))   # alive until wait_host
        return out

    def wait_host(self):
        """Waits for every step_host call of this batch; the host outputs are then complete."""
        _check(load().grace_step_host_wait(self._h), "grace_step_host_wait")
        self._host_pending.clear()

    def flags_check(self, flags) -> int:
        """OR of a device flags array over the batch (synchronises the bound stream)."""
        import torch
        if not (flags.is_cuda and flags.dtype == torch.uint8 and flags.numel() == self.n_cells):
            raise GraceError(f"flags must be a uint8 CUDA tensor of {self.n_cells} elements")
        out = ctypes.c_uint()
        self.ctx.set_stream()
        st = load().grace_flags_check(self._h, _ptr(flags), ctypes.byref(out))
        if st != WARN_CELLS:
            _check(st, "grace_flags_check")
        return out.value

    def mass(self, g):
        import torch
        self._check_state(g)
        m = torch.empty(self.n_cells, dtype=torch.float64, device=g.device)
        self.ctx.set_stream()
        _check(load().grace_mass(self._h, _ptr(g), _ptr(m)), "grace_mass")
        return m

    def limit(self, g, flags=None):
        self._check_state(g)
        self.ctx.set_stream()
        _check(load().grace_limit(self._h, _ptr(g), _ptr(flags)), "grace_limit")
        return g

    def jvp(self, g, v, precision: int = FP64):
        import torch
        self._check_state(g)
        self._check_state(v)
        out = torch.empty_like(g)
        self.ctx.set_stream()
        _check(load().grace_rhs_jvp(self._h, _ptr(g), _ptr(v), _ptr(out), int(precision)), "grace_rhs_jvp")
        return out

    def vjp(self, g, lam, precision: int = FP64):
        import torch
        self._check_state(g)
        self._check_state(lam)
        out = torch.empty_like(g)
        self.ctx.set_stream()
        _check(load().grace_rhs_vjp(self._h, _ptr(g), _ptr(lam), _ptr(out), int(precision)), "grace_rhs_vjp")
        return out

    def adjoint(self, g0, dt, n_steps: int, lam_T, ckpt_every: int = 10, param_grads: bool = False,
                precision: int = FP64):
        """(lambda_0, dtheta [n_cells, n_params] or None) for J with dJ/dg(t_end) = lam_T."""
        import torch
        self._check_state(g0)
        self._check_state(lam_T)
        lam0 = torch.empty_like(g0)
        dth = None
        if param_grads:
            npar = len(getattr(self.ctx, "param_ids", ()))
            dth = torch.zeros(self.n_cells, max(npar, 1), dtype=torch.float64, device=g0.device)
        self.ctx.set_stream()
        _check(load().grace_adjoint(self._h, _ptr(g0), _ptr(dt), int(n_steps), int(ckpt_every), _ptr(lam_T),
                                    _ptr(lam0), _ptr(dth), int(precision)), "grace_adjoint")
        return lam0, dth

    def cell_params(self, alpha):
        """Per-cell alpha_turb for groups with cell_alpha = 1 (device FP64, batch order)."""
        import torch
        a = torch.as_tensor(alpha, dtype=torch.float64, device=f"cuda:{self.ctx.device}").contiguous()
        self.ctx.set_stream()
        _check(load().grace_batch_cell_params(self._h, _ptr(a)), "grace_batch_cell_params")
        self._alpha = a

    def set_graph(self, enable: bool = True):
        """Replay grace_step from a captured CUDA graph for repeated identical calls."""
        _check(load().grace_batch_set_graph(self._h, 1 if enable else 0), "grace_batch_set_graph")

    def set_grouped(self, enable: bool = True):
        """Tensor-form steps of a multi-group batch as one multi-group launch per stage (default)."""
        _check(load().grace_batch_set_grouped(self._h, 1 if enable else 0), "grace_batch_set_grouped")

    def device_error(self) -> int:
        """Reads and clears the device error word (0 = no bounded wait gave up)."""
        code = ctypes.c_int()
        st = load().grace_batch_error(self._h, ctypes.byref(code))
        if st not in (0, 6):
            _check(st, "grace_batch_error")
        return code.value

    def close(self):
        if getattr(self, "_h", None):
            load().grace_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_step_function():
    import torch

    class StepFunction(torch.autograd.Function):
        """g_T = n_steps SSP-RK3 steps (with the limiter) of the batch from g0 in the given form.
        backward runs the checkpointed discrete adjoint (grace_adjoint) in the same form: the
        gradient with respect to g0 and, when theta is given, with respect to the kernel and
        breakage parameters of param_grad_setup (summed over the cells)."""

        @staticmethod
        def forward(ctx, g0, theta, batch, dt, n_steps, ckpt_every, precision):
            g = g0.detach().clone().contiguous()
            batch.step(g, dt, n_steps, precision)
            ctx.batch, ctx.dt, ctx.n_steps, ctx.ckpt, ctx.prec = batch, dt, n_steps, ckpt_every, precision
            ctx.want_theta = theta is not None
            ctx.save_for_backward(g0.detach())
            return g

        @staticmethod
        def backward(ctx, grad_out):
            (g0,) = ctx.saved_tensors
            lam0, dth = ctx.batch.adjoint(g0.contiguous(), ctx.dt, ctx.n_steps, grad_out.contiguous(), ctx.ckpt,
                                          param_grads=ctx.want_theta, precision=ctx.prec)
            gtheta = dth.sum(dim=0) if ctx.want_theta else None
            return lam0, gtheta, None, None, None, None, None

    return StepFunction


def step_autograd(g0, batch, dt, n_steps: int, ckpt_every: int = 10, precision: int = FP64, theta=None):
    """Differentiable wrapper of Batch.step for torch.autograd in any form (FP64, TF32, BF16X3).
    theta: None, or a tensor with one entry per parameter of Context.param_grad_setup (its values
    are not read: the parameters are those of the context); its gradient is dJ/dtheta summed over
    the cells."""
    global StepFunction
    if "StepFunction" not in globals():
        StepFunction = _make_step_function()
    return StepFunction.apply(g0, theta, batch, dt, n_steps, ckpt_every, int(precision))
