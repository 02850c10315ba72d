"""The C ABI library builds, loads and exports every declared entry point
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:dpc_status|int64_t|const\s+char\s*\*)\s*(dpc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = _declared()
    for need in ["dpc_create", "dpc_destroy", "dpc_density", "dpc_dependent", "dpc_label", "dpc_release",
                 "dpc_submit", "dpc_poll", "dpc_last_error"]:
        assert need in names


def test_library_exports_every_declared_symbol():
    import paper_2207_04649_gb300 as dpc
    lib = ctypes.CDLL(dpc.library_path() if os.path.exists(dpc.library_path()) else dpc.lib()._name)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_null_handles_are_rejected_without_a_device():
    import paper_2207_04649_gb300 as dpc
    L = dpc.lib()
    h = ctypes.c_void_p()
    pts = np.zeros((4, 2), np.int32)
    s = L.dpc_density(None, pts.ctypes.data_as(ctypes.c_void_p), 4, 2, 10, 0, ctypes.byref(h), None)
    assert s == dpc.DPC_ERR_INVALID_ARG
    assert "NULL" in dpc.dpc_last_error()
    assert L.dpc_dependent(None, None, None) == dpc.DPC_ERR_STATE
    assert L.dpc_label(None, 1, 2, None, None) == dpc.DPC_ERR_STATE
    assert L.dpc_release(None) == dpc.DPC_ERR_STATE
    assert L.dpc_poll(None, 1, None) == dpc.DPC_ERR_INVALID_ARG
    assert L.dpc_create(None, None) == dpc.DPC_ERR_INVALID_ARG


def test_binding_has_no_cpu_path():
    """The binding never imports the oracle and has no CPU arithmetic."""
    pkg = os.path.join(ROOT, "paper_2207_04649_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "oracle" not in src, f


def test_sapprox_argument_checks_without_a_device():
    import paper_2207_04649_gb300 as dpc
    L = dpc.lib()
    h = ctypes.c_void_p()
    pts = np.zeros((4, 2), np.int32)
    p = pts.ctypes.data_as(ctypes.c_void_p)
    assert L.dpc_sapprox(None, p, 4, 2, 10, 1, 1, 0, ctypes.byref(h), None, None, None, None) == dpc.DPC_ERR_INVALID_ARG
    assert L.dpc_sapprox(ctypes.c_void_p(1), p, 4, 2, 10, 0, 1, 0, ctypes.byref(h), None, None, None, None) \
        == dpc.DPC_ERR_INVALID_ARG
    assert L.dpc_sapprox(ctypes.c_void_p(1), p, 4, 2, 10, 1, (1 << 20) + 1, 0, ctypes.byref(h), None, None, None,
                         None) == dpc.DPC_ERR_INVALID_ARG
    assert "eps" in dpc.dpc_last_error()


def test_eps_fraction():
    import paper_2207_04649_gb300 as dpc
    assert dpc.eps_fraction(0.8) == (4, 5)
    assert dpc.eps_fraction(1.0) == (1, 1)
    assert dpc.eps_fraction((3, 7)) == (3, 7)
    assert dpc.eps_fraction(0.000001) == (1, 1000000)
    with pytest.raises(ValueError):
        dpc.eps_fraction(0.0)


def test_tuning_keys_documented():
    """Every key dpc_set_tuning accepts is documented in the header, and
    every documented key is accepted (read from the sources: no device)."""
    src = open(os.path.join(ROOT, "paper_2207_04649_gb300", "csrc", "runtime.cu")).read()
    accepted = set(re.findall(r'k == "([a-z_0-9]+)"', src))
    doc = open(os.path.join(ROOT, "include", "dpc.h")).read()
    documented = set(re.findall(r'^ \*\s+"([a-z_0-9]+)"', doc, flags=re.M))
    assert accepted and accepted == documented, (accepted ^ documented)


def test_job_footprint_counts_run_slots():
    """The served mode's per-job reservation (host logic, no device):
    n (176 + 8 d + 8 (2R+1)^k) + 16 MB with the default knobs (k = min(d,
    4) gridded dims, reach R = 1 below 7 dims and 2 from 7 on), plus 96 or
    160 bytes per point for the approximate methods' second grid."""
    import paper_2207_04649_gb300 as dpc
    mb16 = 16 << 20
    for d in range(1, 9):
        k = min(d, 4)
        slots = (5 if d >= 7 else 3) ** k
        for n in (0, 1, 1000, 2_000_000):
            base = n * (176 + 8 * d + 8 * slots) + mb16
            assert dpc.dpc_job_footprint(n, d, 0) == base
            assert dpc.dpc_job_footprint(n, d, 1) == base + 96 * n
            assert dpc.dpc_job_footprint(n, d, 2) == base + 160 * n
    # out-of-range arguments are clamped, never negative
    assert dpc.dpc_job_footprint(-5, 3, 0) == mb16
    assert dpc.dpc_job_footprint(10, 0, 0) == dpc.dpc_job_footprint(10, 1, 0)
    assert dpc.dpc_job_footprint(10, 99, 0) == dpc.dpc_job_footprint(10, 8, 0)
