"""ctypes binding of the FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It never touches the CUDA library.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_ubyte)


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("n_bins", ctypes.c_int), ("order_k", ctypes.c_int), ("quad_q", ctypes.c_int),
        ("flux_mode", ctypes.c_int), ("coag_kind", ctypes.c_int), ("frag_kind", ctypes.c_int),
        ("break_kind", ctypes.c_int), ("cutoff_mode", ctypes.c_int), ("limiter", ctypes.c_int),
        ("mfrag_mode", ctypes.c_int),
        ("x_min", ctypes.c_double), ("x_max", ctypes.c_double),
        ("coag_p", ctypes.c_double * 8), ("frag_p", ctypes.c_double * 8),
        ("break_p", ctypes.c_double * 8),
        ("edges", ctypes.POINTER(ctypes.c_double)),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(OrcParams)
        L.orc_gauss.argtypes = [ctypes.c_int, _D, _D]
        L.orc_legendre.argtypes = [ctypes.c_int, ctypes.c_double, _D, _D]
        L.orc_mfrag_ratio.argtypes = [ctypes.c_double]
        L.orc_mfrag_ratio.restype = ctypes.c_double
        L.orc_bin_min.argtypes = [_D, ctypes.c_int]
        L.orc_bin_min.restype = ctypes.c_double
        L.orc_edges.argtypes = [P, _D]
        L.orc_kernels.argtypes = [P, ctypes.c_int, _D, _D, _D, _D]
        L.orc_mass_split.argtypes = [P, ctypes.c_int, _D, _D, _D, _D, _D]
        L.orc_flux_point.argtypes = [P, _D, ctypes.c_int, _D, ctypes.c_int, _D, _D]
        L.orc_vol_frag.argtypes = [P, _D, ctypes.c_int, _D, _D]
        L.orc_appB_pair.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D]
        L.orc_plant_mass_leak.argtypes = [ctypes.c_double]
        L.orc_plant_mass_leak.restype = None
        L.orc_drift_tol.argtypes = [ctypes.c_int]
        L.orc_rhs_species_batch.argtypes = [P, ctypes.c_int, ctypes.c_int, _D, _D, _D]
        L.orc_step_species_batch.argtypes = [P, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_int, _D, _U8]
        L.orc_substep_counts.argtypes = [P, ctypes.c_int, _D, _D, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
        L.orc_drift_tol.restype = ctypes.c_double
        L.orc_rhs_batch.argtypes = [P, ctypes.c_int, _D, _D, _D, ctypes.c_int]
        L.orc_limit_batch.argtypes = [P, ctypes.c_int, _D, _U8]
        L.orc_step_batch.argtypes = [P, ctypes.c_int, _D, _D, ctypes.c_int, _D, _U8, ctypes.c_int]
        L.orc_mass_batch.argtypes = [P, ctypes.c_int, _D, _D]
        L.orc_project_batch.argtypes = [P, ctypes.c_int, ctypes.c_int, _D, _D]
        L.orc_max_threads.restype = ctypes.c_int
        L.orc_tangent_rhs.argtypes = [P, ctypes.c_int, _D, _D, ctypes.c_int, _D, _D]
        L.orc_tangent_step.argtypes = [P, ctypes.c_int, _D, _D, ctypes.c_int, _D, ctypes.c_int, _D, _D]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def params(spec) -> OrcParams:
    p = OrcParams()
    p.n_bins, p.order_k, p.quad_q = spec.n_bins, spec.order_k, spec.quad_q
    p.flux_mode, p.coag_kind, p.frag_kind = spec.flux_mode, spec.coag_kind, spec.frag_kind
    p.break_kind, p.cutoff_mode, p.limiter = spec.break_kind, spec.cutoff_mode, spec.limiter
    p.mfrag_mode = spec.mfrag_mode
    p.x_min, p.x_max = spec.x_min, spec.x_max
    for name in ("coag_p", "frag_p", "break_p"):
        vals = getattr(spec, name)
        arr = getattr(p, name)
        for i, v in enumerate(vals):
            arr[i] = v
    if getattr(spec, "edges", None) is not None:
        buf = (ctypes.c_double * len(spec.edges))(*spec.edges)
        p.edges = ctypes.cast(buf, _D)
        p._edges_buf = buf          # alive as long as the parameter block
    return p


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def gauss(Q: int):
    s = np.zeros(Q)
    w = np.zeros(Q)
    _check(lib().orc_gauss(Q, _p(s), _p(w)), "gauss")
    return s, w


def legendre(k: int, xi: float):
    P = np.zeros(k + 1)
    dP = np.zeros(k + 1)
    _check(lib().orc_legendre(k, float(xi), _p(P), _p(dP)), "legendre")
    return P, dP


def mfrag_ratio(q: float) -> float:
    return lib().orc_mfrag_ratio(float(q))


def bin_min(gj, k: int) -> float:
    gj = _f64(gj)
    return lib().orc_bin_min(_p(gj), int(k))


def plant_mass_leak(leak: float) -> None:
    """Plants a non-conservative update (leak * M_1 added to bin 0 every step) in every later
    oracle step; 0 removes it.  For tests of the mass-drift bit only."""
    lib().orc_plant_mass_leak(float(leak))


def drift_tol(n_steps: int) -> float:
    """Relative M_1 change above which a call of n_steps steps sets the mass-drift bit."""
    return lib().orc_drift_tol(int(n_steps))


def max_threads() -> int:
    return lib().orc_max_threads()


class Oracle:
    """FP64 reference for one group description (see paper_2607_13740_b300.workloads.GroupSpec)."""

    def __init__(self, spec):
        self.spec = spec
        self._par = params(spec)
        self.P = spec.n_bins * (spec.order_k + 1)

    @property
    def _pp(self):
        return ctypes.byref(self._par)

    def edges(self):
        e = np.zeros(self.spec.n_bins + 1)
        _check(lib().orc_edges(self._pp, _p(e)), "edges")
        return e

    def kernels(self, u, v):
        u, v = _f64(u), _f64(v)
        kc, kf = np.zeros_like(u), np.zeros_like(u)
        _check(lib().orc_kernels(self._pp, u.size, _p(u), _p(v), _p(kc), _p(kf)), "kernels")
        return kc, kf

    def mass_split(self, x, u, v):
        x, u, v = _f64(x), _f64(u), _f64(v)
        a, b = np.zeros_like(x), np.zeros_like(x)
        _check(lib().orc_mass_split(self._pp, x.size, _p(x), _p(u), _p(v), _p(a), _p(b)), "mass_split")
        return a, b

    def flux_point(self, g, x, parts: int = 3):
        g = _f64(g).reshape(-1)
        x = _f64(np.atleast_1d(x))
        F, Fa = np.zeros_like(x), np.zeros_like(x)
        _check(lib().orc_flux_point(self._pp, _p(g), x.size, _p(x), parts, _p(F), _p(Fa)), "flux_point")
        return F, Fa

    def vol_frag(self, g, j: int):
        g = _f64(g).reshape(-1)
        V = np.zeros(self.spec.order_k + 1)
        Va = np.zeros_like(V)
        _check(lib().orc_vol_frag(self._pp, _p(g), int(j), _p(V), _p(Va)), "vol_frag")
        return V, Va

    def appB_pair(self, j: int, u: float, v: float):
        """App. B sub-interval integrals of one collision pair (u, v) in bin j: J[i], i = 0..k."""
        J = np.zeros(self.spec.order_k + 1)
        _check(lib().orc_appB_pair(self._pp, int(j), float(u), float(v), _p(J)), "appB_pair")
        return J

    def rhs_species(self, gs):
        """Species of mixed grains (Sec. 5.3): gs [S, n_cells, P] partial mass densities; returns
        (L_s, S_s) in the same layout, L_s = L[g_s; sum_s g_s] (the species in the outer slot)."""
        gs = np.ascontiguousarray(gs, dtype=np.float64)
        S_, n = gs.shape[0], gs.shape[1]
        L = np.zeros_like(gs)
        Sc = np.zeros_like(gs)
        _check(lib().orc_rhs_species_batch(self._pp, n, S_, _p(gs), _p(L), _p(Sc)), "rhs_species")
        return L, Sc

    def step_species(self, gs, dt, n_steps: int):
        """n_steps SSP-RK3 steps of the species [S, n_cells, P]; returns (gs, mass [S, n_cells], flags)."""
        gs = np.ascontiguousarray(gs, dtype=np.float64).copy()
        S_, n = gs.shape[0], gs.shape[1]
        dt = _f64(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)))
        mass = np.zeros((S_, n))
        f = np.zeros(n, dtype=np.uint8)
        _check(lib().orc_step_species_batch(self._pp, n, S_, _p(gs), _p(dt), int(n_steps), _p(mass),
                                            f.ctypes.data_as(_U8)), "step_species")
        return gs, mass, f

    def tangent_rhs(self, g, gdot=None, param_id: int = -1):
        """Forward-mode derivative build: returns (L[g], dL) with dL the exact derivative of the
        oracle's L along gdot (None: zero) and parameter param_id (0..7 coag_p, 8..15 frag_p,
        16..23 break_p; -1 none)."""
        g = _f64(g).reshape(-1, self.P)
        gd = None if gdot is None else _f64(gdot).reshape(g.shape)
        L = np.zeros_like(g)
        dL = np.zeros_like(g)
        _check(lib().orc_tangent_rhs(self._pp, g.shape[0], _p(g), None if gd is None else _p(gd), int(param_id),
                                     _p(L), _p(dL)), "tangent_rhs")
        return L, dL

    def tangent_step(self, g, dt, n_steps: int, gdot=None, param_id: int = -1):
        """n_steps oracle steps (limiter + SSP-RK3) on dual numbers: returns (g(T), dg(T)), the
        exact derivative of the final state along gdot and parameter param_id."""
        g = _f64(g).reshape(-1, self.P)
        n = g.shape[0]
        gd = None if gdot is None else _f64(gdot).reshape(g.shape)
        dt = _f64(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)))
        out = np.zeros_like(g)
        dout = np.zeros_like(g)
        _check(lib().orc_tangent_step(self._pp, n, _p(g), None if gd is None else _p(gd), int(param_id), _p(dt),
                                      int(n_steps), _p(out), _p(dout)), "tangent_step")
        return out, dout

    def substep_counts(self, g, dt_hydro, cfl: float):
        """Per-cell sub-step counts ceil(dt_hydro / (cfl B)) of the operator-split coupling, B the eq. (dt)
        bound of the state (Sec. 5.2)."""
        g = _f64(g).reshape(-1, self.P)
        dt = _f64(np.broadcast_to(np.asarray(dt_hydro, dtype=np.float64), (g.shape[0],)))
        out = np.zeros(g.shape[0], dtype=np.int32)
        _check(lib().orc_substep_counts(self._pp, g.shape[0], _p(g), _p(dt), float(cfl),
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_int))), "substep_counts")
        return out

    def substep(self, g, dt_hydro, cfl: float, max_substeps: int, threads: int = 0):
        """The batch's operator-split step: N = min(max counts, max_substeps) SSP-RK3 steps of
        dt_hydro / N per cell.  Returns (g, mass, flags, N)."""
        counts = self.substep_counts(g, dt_hydro, cfl)
        N = int(max(1, min(int(counts.max()), int(max_substeps))))
        dt = np.broadcast_to(np.asarray(dt_hydro, dtype=np.float64), (counts.size,)) / N
        g2, m, f = self.step(g, dt, N, threads=threads)
        return g2, m, f, N

    def rhs(self, g, threads: int = 0):
        g = _f64(g).reshape(-1, self.P)
        L = np.zeros_like(g)
        S = np.zeros_like(g)
        _check(lib().orc_rhs_batch(self._pp, g.shape[0], _p(g), _p(L), _p(S), threads), "rhs")
        return L, S

    def limit(self, g):
        g = _f64(g).reshape(-1, self.P).copy()
        f = np.zeros(g.shape[0], dtype=np.uint8)
        _check(lib().orc_limit_batch(self._pp, g.shape[0], _p(g), f.ctypes.data_as(_U8)), "limit")
        return g, f

    def step(self, g, dt, n_steps: int, threads: int = 0):
        g = _f64(g).reshape(-1, self.P).copy()
        n = g.shape[0]
        dt = _f64(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)))
        mass = np.zeros(n)
        f = np.zeros(n, dtype=np.uint8)
        _check(lib().orc_step_batch(self._pp, n, _p(g), _p(dt), int(n_steps), _p(mass),
                                    f.ctypes.data_as(_U8), threads), "step")
        return g, mass, f

    def mass(self, g):
        g = _f64(g).reshape(-1, self.P)
        m = np.zeros(g.shape[0])
        _check(lib().orc_mass_batch(self._pp, g.shape[0], _p(g), _p(m)), "mass")
        return m

    def project(self, ic_kind: int, ic_params):
        ic = _f64(np.atleast_2d(ic_params))
        if ic.shape[1] < 4:
            ic = np.pad(ic, ((0, 0), (0, 4 - ic.shape[1])))
        g = np.zeros((ic.shape[0], self.P))
        _check(lib().orc_project_batch(self._pp, ic.shape[0], int(ic_kind), _p(ic), _p(g)), "project")
        return g


# ---------------------------------------------------------------- two dimensions (mass, volume)
class MVDesc(ctypes.Structure):
    _fields_ = [
        ("Nx", ctypes.c_int), ("Nv", ctypes.c_int), ("k", ctypes.c_int), ("Q", ctypes.c_int),
        ("x_min", ctypes.c_double), ("x_max", ctypes.c_double), ("v_min", ctypes.c_double),
        ("v_max", ctypes.c_double), ("n_terms", ctypes.c_int),
        ("coef", ctypes.c_double * 8), ("ax", ctypes.c_double * 8), ("bx", ctypes.c_double * 8),
        ("av", ctypes.c_double * 8), ("bv", ctypes.c_double * 8),
    ]


def mv_desc(spec) -> MVDesc:
    d = MVDesc()
    d.Nx, d.Nv, d.k, d.Q = spec.n_x, spec.n_v, spec.order_k, spec.quad_q
    d.x_min, d.x_max, d.v_min, d.v_max = spec.x_min, spec.x_max, spec.v_min, spec.v_max
    d.n_terms = len(spec.terms)
    for t, (c, ax, bx, av, bv) in enumerate(spec.terms):
        d.coef[t], d.ax[t], d.bx[t], d.av[t], d.bv[t] = c, ax, bx, av, bv
    return d


class MVOracle:
    """The two-dimensional (mass, volume) weak form of Sec. 5.3 (grace_oracle_mv.c)."""

    def __init__(self, spec):
        self.spec = spec
        self.d = mv_desc(spec)
        L = lib()
        P = ctypes.POINTER(MVDesc)
        L.orc_mv_rhs.argtypes = [P, ctypes.c_int, _D, _D]
        L.orc_mv_step.argtypes = [P, ctypes.c_int, _D, _D, ctypes.c_int]
        L.orc_mv_mass.argtypes = [P, ctypes.c_int, _D, _D]
        L.orc_mv_edges.argtypes = [P, _D, _D]

    def rhs(self, g):
        g = _f64(g).reshape(-1, self.spec.n_coef)
        L = np.zeros_like(g)
        _check(lib().orc_mv_rhs(ctypes.byref(self.d), g.shape[0], _p(g), _p(L)), "mv rhs")
        return L

    def step(self, g, dt, n_steps):
        g = _f64(g).reshape(-1, self.spec.n_coef).copy()
        dt = _f64(np.broadcast_to(dt, (g.shape[0],)))
        _check(lib().orc_mv_step(ctypes.byref(self.d), g.shape[0], _p(g), _p(dt), int(n_steps)), "mv step")
        return g

    def mass(self, g):
        g = _f64(g).reshape(-1, self.spec.n_coef)
        m = np.zeros(g.shape[0])
        _check(lib().orc_mv_mass(ctypes.byref(self.d), g.shape[0], _p(g), _p(m)), "mv mass")
        return m

    def edges(self):
        ex = np.zeros(self.spec.n_x + 1)
        ev = np.zeros(self.spec.n_v + 1)
        _check(lib().orc_mv_edges(ctypes.byref(self.d), _p(ex), _p(ev)), "mv edges")
        return ex, ev
