"""Host-side checks of the C-ABI library: it loads, exports every declared
symbol, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import numpy as np

import pytest

from paper_2607_13740_b300 import build, grace, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "grace.h")).read()
    return sorted(set(re.findall(r"GRACE_API[^;(]*?\b(grace_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return grace.load()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 16
    raw = ctypes.CDLL(grace.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n
    assert set(grace.exported_symbols()) <= set(names)


def test_version_and_status_strings(lib):
    assert lib.grace_version() >= 1
    for s in range(0, 7):
        assert lib.grace_status_string(s).decode()
    assert lib.grace_status_string(99).decode() == "unknown status"


def _setup(lib, desc, n=1, device=0):
    h = ctypes.c_void_p()
    arr = (grace.GroupDesc * n)(*([desc] * n))
    return lib.grace_setup(ctypes.byref(h), n, arr, device), h


@pytest.mark.parametrize("field,value", [
    ("n_bins", 1), ("order_k", -1), ("quad_q", 17), ("x_min", 0.0), ("x_max", 1e-9),
    ("flux_mode", 2), ("coag_kind", 9), ("frag_kind", 7), ("break_kind", 5), ("limiter", 3),
])
def test_setup_rejects_invalid_groups(lib, field, value):
    d = grace.group_desc(W.additive_spec(8, 2))
    setattr(d, field, value)
    st, h = _setup(lib, d)
    assert st == 1, lib.grace_last_error()
    assert not h.value
    assert lib.grace_last_error().decode()


def test_setup_reports_unsupported_order(lib):
    """k <= 4 (the limiter's bin minimum: closed form to k = 3, bracketed for k = 4); per-cell
    kernel groups k <= 3 (node-space entry layout)."""
    d = grace.group_desc(W.additive_spec(8, 5))
    st, _ = _setup(lib, d)
    assert st == 5
    d = grace.group_desc(W.disk_spec(n_bins=8, order_k=4))
    st, _ = _setup(lib, d)
    assert st == 1


def test_setup_rejects_missing_kernels_and_bad_power_law(lib):
    d = grace.group_desc(W.additive_spec(8, 2).replace(coag_kind=W.COAG_NONE))
    assert _setup(lib, d)[0] == 1
    d = grace.group_desc(W.coupled_toy_spec(8, 2).replace(break_p=(-2.0,)))
    assert _setup(lib, d)[0] == 1


def test_null_arguments_are_errors(lib):
    assert lib.grace_setup(None, 1, None, 0) == 1
    assert lib.grace_set_stream(None, None) == 1
    assert lib.grace_precompute(None, 0) == 1
    assert lib.grace_bind_batch(None, 4, None, None) == 1
    assert lib.grace_rhs(None, None, None, 0) == 1
    assert lib.grace_step(None, None, None, 1, 0, None, None) == 1
    assert lib.grace_mass(None, None, None) == 1
    lib.grace_batch_destroy(None)
    lib.grace_destroy(None)


def test_negative_device_is_rejected_on_host(lib):
    d = grace.group_desc(W.additive_spec(8, 2))
    assert _setup(lib, d, device=-1)[0] == 1


def test_host_step_rejects_null_batch(lib):
    """grace_step_host / grace_step_host_wait check their arguments before any CUDA call."""
    buf = (ctypes.c_double * 4)()
    assert lib.grace_step_host(None, buf, buf, buf, 1, 0, None, None) == 1
    assert lib.grace_step_host_wait(None) == 1
    assert "grace_step_host" in lib.grace_last_error().decode()


def test_flags_check_rejects_null_and_names_warn_status(lib):
    assert lib.grace_flags_check(None, None, None) == 1
    assert lib.grace_status_string(grace.WARN_CELLS).decode() != "unknown status"


def test_binding_fails_loudly_without_the_library():
    """No CPU fallback: without the built CUDA library the binding raises."""
    import subprocess
    import sys
    code = ("from paper_2607_13740_b300 import grace\n"
            "grace.load('" + os.path.join(ROOT, "_missing", "libgrace.so") + "')\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert out.returncode != 0
    assert "CUDA library not built" in out.stderr


def test_set_cta_pairs_accepts_only_its_three_modes():
    for v in (0, 1, 2):
        grace.set_cta_pairs(v)
    for bad in (-1, 3):
        with pytest.raises(grace.GraceError):
            grace.set_cta_pairs(bad)
    grace.set_cta_pairs(grace.CTA_PAIRS_NEVER)


def test_set_tc_a_in_tmem_accepts_only_zero_and_one():
    grace.set_tc_a_in_tmem(True)
    grace.set_tc_a_in_tmem(False)
    for bad in (-1, 2):
        with pytest.raises(grace.GraceError):
            grace._check(grace.load().grace_set_tc_a_in_tmem(bad), "grace_set_tc_a_in_tmem")


def test_arm_wait_timeout_rejects_bad_limits():
    """The failure-detection hook takes limits in [1, 4e9] cycles only (no GPU needed)."""
    with pytest.raises(grace.GraceError):
        grace.arm_wait_timeout(0)
    with pytest.raises(grace.GraceError):
        grace.arm_wait_timeout(5_000_000_000)


@pytest.mark.parametrize("bad", ["decreasing", "ends", "nan"])
def test_setup_rejects_invalid_edges(lib, bad):
    """Caller-supplied bin edges are validated on the host before any CUDA call."""
    spec = W.additive_spec(6, 1, 1e-2, 1e2)
    e = list(spec.x_min * (spec.x_max / spec.x_min) ** (np.arange(7) / 6))
    e[0], e[-1] = spec.x_min, spec.x_max
    if bad == "decreasing":
        e[2], e[3] = e[3], e[2]
    elif bad == "ends":
        e[-1] = 2e2
    else:
        e[4] = float("nan")
    d = grace.group_desc(spec.replace(edges=tuple(e)))
    st, h = _setup(lib, d)
    assert st == 1 and not h.value
    assert "edges" in lib.grace_last_error().decode()


@pytest.mark.parametrize("field,value", [("n_x", 0), ("n_v", 0), ("order_k", 5), ("quad_q", 0), ("quad_q", 25),
                                         ("x_min", 0.0), ("v_max", 1e-3), ("n_terms", 0), ("n_terms", 9),
                                         ("arithmetic", 2), ("arithmetic", -1)])
def test_mv_setup_rejects_invalid_descriptions(field, value):
    """The two-dimensional setup validates its description on the host (no GPU needed)."""
    from paper_2607_13740_b300 import workloads as W
    d = grace.mv_desc(W.mv_mixed_spec())
    setattr(d, field, value)
    h = ctypes.c_void_p()
    assert grace.load().grace_mv_setup(ctypes.byref(h), ctypes.byref(d), 0) == 1   # GRACE_ERR_ARG
    assert not h.value


def test_mv_setup_rejects_non_finite_kernel_terms():
    from paper_2607_13740_b300 import workloads as W
    d = grace.mv_desc(W.mv_mixed_spec())
    d.coef[0] = float("nan")
    h = ctypes.c_void_p()
    assert grace.load().grace_mv_setup(ctypes.byref(h), ctypes.byref(d), 0) == 1
    assert grace.load().grace_mv_rhs(None, 1, None, None) == 1
    assert grace.load().grace_mv_step(None, 1, None, None, 1) == 1
