"""CPU oracle for exact Density-Peaks Clustering.

TEST INFRASTRUCTURE. This package is the plain, slow reference the CUDA
library is checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the library itself never
does, and it shares no code with the library.

The arithmetic lives in ``dpc_oracle.c`` (plain C with OpenMP over points,
built here with gcc); this module compiles it and wraps it with numpy. Every
function follows the paper's problem definition (Section 2.1, Definitions
1-6) and its straightforward Scan algorithm (Section 2.2); the ``approx_*``
functions follow Approx-DPC's dependent-point rules (Section 4.3); the
``sapprox*`` functions follow S-Approx-DPC (Section 5). The readings of the
paper it takes are listed in ``dpc_oracle.c``.

Parity status: every function is pinned by the tests in
``tests/test_oracle.py``, ``tests/test_oracle_approx.py`` and
``tests/test_oracle_sapprox.py`` (hand-worked examples in ``tests/golden/``,
closed forms, invariants, an independent brute force, the paper's
cluster-center guarantee for Approx-DPC, S-Approx-DPC reducing to exact DPC
on cells of one point, and planted mistakes), so none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

INT64_MAX = np.iinfo(np.int64).max


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        vp = ctypes.c_void_p
        lib.oracle_threads.restype = ctypes.c_int
        lib.oracle_rho.argtypes = [vp, i64, i32, i64, vp]
        lib.oracle_rho_subset.argtypes = [vp, i64, i32, i64, vp, i64, vp]
        lib.oracle_rank_order.argtypes = [vp, i64, vp]
        lib.oracle_dependent.argtypes = [vp, i64, i32, vp, vp, vp]
        lib.oracle_dependent_subset.argtypes = [vp, i64, i32, vp, vp, i64, vp, vp]
        lib.oracle_label.argtypes = [i64, vp, vp, vp, i64, i64, vp]
        lib.oracle_label.restype = i64
        lib.oracle_approx_side.argtypes = [i64, i32]
        lib.oracle_approx_side.restype = i64
        lib.oracle_approx_dependent.argtypes = [vp, i64, i32, i64, vp, vp, vp, vp]
        lib.oracle_approx_dependent_subset.argtypes = [vp, i64, i32, i64, vp, vp, i64, vp, vp, vp]
        lib.oracle_sapprox_side.argtypes = [i64, i32, i64, i64]
        lib.oracle_sapprox_side.restype = i64
        lib.oracle_sapprox.argtypes = [vp, i64, i32, i64, i64, i64, vp, vp, vp, vp]
        lib.oracle_sapprox_dependent_subset.argtypes = [vp, i64, i32, i64, i64, i64, vp, vp, i64, vp, vp, vp]
        lib.oracle_sapprox_label.argtypes = [i64, vp, vp, vp, vp, i64, i64, vp]
        lib.oracle_sapprox_label.restype = i64
        _lib = lib
        return lib


def _pts(points) -> np.ndarray:
    p = np.ascontiguousarray(points, dtype=np.int32)
    if p.ndim != 2:
        raise ValueError("points must be an n x d array")
    return p


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    """Number of OpenMP threads the oracle runs on."""
    return int(_load().oracle_threads())


def rho(points, d_cut: int) -> np.ndarray:
    """Definition 1: rho_i = #{j : D(i,j) < d_cut^2}, p_i included."""
    p = _pts(points)
    n, d = p.shape
    out = np.empty(n, dtype=np.int32)
    _load().oracle_rho(_ptr(p), n, d, int(d_cut), _ptr(out))
    return out


def rho_subset(points, d_cut: int, idx) -> np.ndarray:
    """Definition 1 for the points listed in ``idx`` (each against all n)."""
    p = _pts(points)
    n, d = p.shape
    ix = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(ix.shape[0], dtype=np.int32)
    _load().oracle_rho_subset(_ptr(p), n, d, int(d_cut), _ptr(ix), ix.shape[0], _ptr(out))
    return out


def rank_order(rho_arr) -> np.ndarray:
    """Scan step 2: indices sorted by (rho desc, index asc)."""
    r = np.ascontiguousarray(rho_arr, dtype=np.int32)
    out = np.empty(r.shape[0], dtype=np.int64)
    _load().oracle_rank_order(_ptr(r), r.shape[0], _ptr(out))
    return out


def dependent(points, rho_arr):
    """Scan step 3 / Definitions 2-3: (dep int32, delta2 int64)."""
    p = _pts(points)
    n, d = p.shape
    r = np.ascontiguousarray(rho_arr, dtype=np.int32)
    dep = np.empty(n, dtype=np.int32)
    d2 = np.empty(n, dtype=np.int64)
    _load().oracle_dependent(_ptr(p), n, d, _ptr(r), _ptr(dep), _ptr(d2))
    return dep, d2


def dependent_subset(points, rho_arr, idx):
    """Definitions 2-3 for the points in ``idx`` against every higher point."""
    p = _pts(points)
    n, d = p.shape
    r = np.ascontiguousarray(rho_arr, dtype=np.int32)
    ix = np.ascontiguousarray(idx, dtype=np.int64)
    dep = np.empty(ix.shape[0], dtype=np.int32)
    d2 = np.empty(ix.shape[0], dtype=np.int64)
    _load().oracle_dependent_subset(_ptr(p), n, d, _ptr(r), _ptr(ix), ix.shape[0],
                                    _ptr(dep), _ptr(d2))
    return dep, d2


def label(rho_arr, dep, delta2, rho_min: int, delta_min: int):
    """Scan step 4 / Definitions 4-6: (label int32, n_centers)."""
    r = np.ascontiguousarray(rho_arr, dtype=np.int32)
    dp = np.ascontiguousarray(dep, dtype=np.int32)
    d2 = np.ascontiguousarray(delta2, dtype=np.int64)
    n = r.shape[0]
    lab = np.empty(n, dtype=np.int32)
    nc = _load().oracle_label(n, _ptr(r), _ptr(dp), _ptr(d2), int(rho_min), int(delta_min),
                              _ptr(lab))
    return lab, int(nc)


def approx_side(d_cut: int, d: int) -> int:
    """Approx-DPC's grid side: max(1, floor(d_cut / sqrt(d)))."""
    return int(_load().oracle_approx_side(int(d_cut), int(d)))


def approx_dependent(points, rho_arr, d_cut: int):
    """Approx-DPC's dependent points (Section 4.3): (dep, delta2, exact) where
    exact marks the points whose dependent point was computed exactly."""
    p = _pts(points)
    n, d = p.shape
    r = np.ascontiguousarray(rho_arr, dtype=np.int32)
    dep = np.empty(n, dtype=np.int32)
    d2 = np.empty(n, dtype=np.int64)
    ex = np.empty(n, dtype=np.int32)
    _load().oracle_approx_dependent(_ptr(p), n, d, int(d_cut), _ptr(r), _ptr(dep), _ptr(d2), _ptr(ex))
    return dep, d2, ex.astype(bool)


def approx_dependent_subset(points, rho_arr, d_cut: int, idx):
    """Approx-DPC's dependent points of the points listed in ``idx``."""
    p = _pts(points)
    n, d = p.shape
    r = np.ascontiguousarray(rho_arr, dtype=np.int32)
    ix = np.ascontiguousarray(idx, dtype=np.int64)
    m = ix.shape[0]
    dep = np.empty(m, dtype=np.int32)
    d2 = np.empty(m, dtype=np.int64)
    ex = np.empty(m, dtype=np.int32)
    _load().oracle_approx_dependent_subset(_ptr(p), n, d, int(d_cut), _ptr(r), _ptr(ix), m, _ptr(dep), _ptr(d2),
                                           _ptr(ex))
    return dep, d2, ex.astype(bool)


def run_approx(points, d_cut: int, rho_min: int, delta_min: int) -> dict:
    """Approx-DPC: exact rho, approximate dependent points, labels."""
    r = rho(points, d_cut)
    dep, d2, ex = approx_dependent(points, r, d_cut)
    lab, nc = label(r, dep, d2, rho_min, delta_min)
    return {"rho": r, "dep": dep, "delta2": d2, "exact": ex, "label": lab, "n_centers": nc}


def sapprox_side(d_cut: int, d: int, eps_num: int, eps_den: int) -> int:
    """S-Approx-DPC's grid side: max(1, floor(eps d_cut / sqrt(d))), eps = num / den."""
    return int(_load().oracle_sapprox_side(int(d_cut), int(d), int(eps_num), int(eps_den)))


def sapprox(points, d_cut: int, eps_num: int, eps_den: int):
    """S-Approx-DPC (Section 5): (rho, dep, delta2, pick); rho is -1 and dep
    the cell's pick for the points that are not picked."""
    p = _pts(points)
    n, d = p.shape
    rho_ = np.empty(n, dtype=np.int32)
    dep = np.empty(n, dtype=np.int32)
    d2 = np.empty(n, dtype=np.int64)
    pk = np.empty(n, dtype=np.int32)
    _load().oracle_sapprox(_ptr(p), n, d, int(d_cut), int(eps_num), int(eps_den), _ptr(rho_), _ptr(dep), _ptr(d2),
                           _ptr(pk))
    return rho_, dep, d2, pk.astype(bool)


def sapprox_dependent_subset(points, rho_arr, d_cut: int, eps_num: int, eps_den: int, idx):
    """Sampled S-Approx-DPC links: (dep, delta2, pick) of the points idx,
    given rho of every pick (other entries unused)."""
    p = _pts(points)
    n, d = p.shape
    r = np.ascontiguousarray(rho_arr, dtype=np.int32)
    ix = np.ascontiguousarray(idx, dtype=np.int64)
    m = ix.shape[0]
    dep = np.empty(m, dtype=np.int32)
    d2 = np.empty(m, dtype=np.int64)
    pk = np.empty(m, dtype=np.int32)
    _load().oracle_sapprox_dependent_subset(_ptr(p), n, d, int(d_cut), int(eps_num), int(eps_den), _ptr(r), _ptr(ix),
                                            m, _ptr(dep), _ptr(d2), _ptr(pk))
    return dep, d2, pk.astype(bool)


def sapprox_label(rho_arr, dep, delta2, pick, rho_min: int, delta_min: int):
    """S-Approx-DPC labels: Definitions 4-6 over the picks, others take their pick's label."""
    r = np.ascontiguousarray(rho_arr, dtype=np.int32)
    dp = np.ascontiguousarray(dep, dtype=np.int32)
    d2 = np.ascontiguousarray(delta2, dtype=np.int64)
    pk = np.ascontiguousarray(pick, dtype=np.int32)
    n = r.shape[0]
    lab = np.empty(n, dtype=np.int32)
    nc = _load().oracle_sapprox_label(n, _ptr(r), _ptr(dp), _ptr(d2), _ptr(pk), int(rho_min), int(delta_min),
                                      _ptr(lab))
    return lab, int(nc)


def run(points, d_cut: int, rho_min: int, delta_min: int) -> dict:
    """The whole path: rho, dependent point, squared delta, labels."""
    r = rho(points, d_cut)
    dep, d2 = dependent(points, r)
    lab, nc = label(r, dep, d2, rho_min, delta_min)
    return {"rho": r, "dep": dep, "delta2": d2, "label": lab, "n_centers": nc}
