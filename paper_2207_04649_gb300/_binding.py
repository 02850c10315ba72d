"""ctypes binding of libdpc (argument marshalling only).

Host data is passed as numpy arrays, device data as CUDA torch tensors (their
data pointers). PyTorch is used for device memory and streams only.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

DPC_OK = 0
DPC_PENDING = 1
DPC_ERR_INVALID_ARG = -1
DPC_ERR_OOM = -2
DPC_ERR_CUDA = -3
DPC_ERR_TIMEOUT = -4
DPC_ERR_STATE = -5
DPC_ERR_CAPACITY = -6
INT64_MAX = np.iinfo(np.int64).max

_NAMES = {0: "DPC_OK", 1: "DPC_PENDING", -1: "DPC_ERR_INVALID_ARG", -2: "DPC_ERR_OOM", -3: "DPC_ERR_CUDA",
          -4: "DPC_ERR_TIMEOUT", -5: "DPC_ERR_STATE", -6: "DPC_ERR_CAPACITY"}


class DpcError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {_NAMES.get(status, status)}: {msg}")
        self.status = status


class DpcOptions(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("hbm_cap_bytes", ctypes.c_uint64),
                ("tune_cache", ctypes.c_char_p), ("debug_checks", ctypes.c_int), ("mode", ctypes.c_int),
                ("max_inflight", ctypes.c_int)]


class DpcInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("cells", ctypes.c_int64), ("dense_cells", ctypes.c_int64),
                ("work_items", ctypes.c_int64), ("cand_pairs", ctypes.c_int64),
                ("open_after_ring", ctypes.c_int64), ("brute_points", ctypes.c_int64),
                ("grid_dims", ctypes.c_int32), ("pair_bits", ctypes.c_int32),
                ("ms_grid", ctypes.c_float), ("ms_rho", ctypes.c_float), ("ms_rank", ctypes.c_float),
                ("ms_ring", ctypes.c_float), ("ms_rest", ctypes.c_float), ("ms_label", ctypes.c_float),
                ("tree_visits", ctypes.c_int64), ("tree_pairs", ctypes.c_int64),
                ("pair_mode", ctypes.c_int32), ("grid_key_bits", ctypes.c_int32),
                ("dense_pairs", ctypes.c_int64), ("ms_rho_dense", ctypes.c_float), ("rank_key_bits", ctypes.c_int32),
                ("picks", ctypes.c_int64), ("second_phase", ctypes.c_int64), ("density_path", ctypes.c_int32),
                ("device_bytes_peak", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class DpcJob(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32),
                ("d_cut", ctypes.c_int64), ("n_queries", ctypes.c_int32), ("rho_min", ctypes.c_void_p),
                ("delta_min", ctypes.c_void_p), ("rho_out", ctypes.c_void_p), ("dep_out", ctypes.c_void_p),
                ("delta2_out", ctypes.c_void_p), ("label_out", ctypes.c_void_p),
                ("n_centers_out", ctypes.c_void_p), ("is_device", ctypes.c_int32), ("method", ctypes.c_int32),
                ("eps_num", ctypes.c_int64), ("eps_den", ctypes.c_int64), ("aux_out", ctypes.c_void_p),
                ("keep", ctypes.c_int32)]

METHODS = {"exact": 0, "approx": 1, "sapprox": 2}


class DpcResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("dataset", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libdpc.so, building it first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        L = ctypes.CDLL(path)
        vp, i64, i32, st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        sig = {
            "dpc_create": ([ctypes.POINTER(DpcOptions), ctypes.POINTER(vp)], st),
            "dpc_destroy": ([vp], st),
            "dpc_last_error": ([], ctypes.c_char_p),
            "dpc_density": ([vp, vp, i64, i32, i64, ctypes.c_int, ctypes.POINTER(vp), vp], st),
            "dpc_dependent": ([vp, vp, vp], st),
            "dpc_label": ([vp, i64, i64, vp, ctypes.POINTER(i64)], st),
            "dpc_release": ([vp], st),
            "dpc_ds_info": ([vp, ctypes.POINTER(DpcInfo)], st),
            "dpc_last_batch_info": ([vp, ctypes.POINTER(DpcInfo)], st),
            "dpc_dependent_approx": ([vp, vp, vp, vp], st),
            "dpc_cluster": ([vp, vp, i64, i32, i64, ctypes.c_int, i64, i64, vp, vp, vp, vp, ctypes.POINTER(i64)], st),
            "dpc_sapprox": ([vp, vp, i64, i32, i64, i64, i64, ctypes.c_int, ctypes.POINTER(vp), vp, vp, vp, vp], st),
            "dpc_autotune": ([vp, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_char_p,
                              ctypes.c_size_t], st),
            "dpc_set_profiling": ([vp, ctypes.c_int], st),
            "dpc_submit": ([vp, ctypes.POINTER(DpcJob), ctypes.POINTER(ctypes.c_uint64)], st),
            "dpc_poll": ([vp, ctypes.c_uint64, ctypes.POINTER(DpcResult)], st),
            "dpc_flush": ([vp], st),
            "dpc_wait": ([vp, ctypes.c_uint64, i64, ctypes.POINTER(DpcResult)], st),
            "dpc_kernel_launches": ([], i64),
            "dpc_job_footprint": ([vp, i64, i32, i32], ctypes.c_uint64),
            "dpc_set_tuning": ([vp, ctypes.c_char_p, i64], st),
            "dpc_get_tuning": ([vp, ctypes.c_char_p, ctypes.POINTER(i64)], st),
            "dpc_probe_pair_rate": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)], st),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return L


def dpc_kernel_launches() -> int:
    return int(lib().dpc_kernel_launches())


def dpc_job_footprint(n: int, d: int, method: int = 0, ctx=None) -> int:
    """Device bytes the served mode reserves for a job of n points in d dims
    (method 0 exact, 1 Approx-DPC, 2 S-Approx-DPC) under ctx's tuning knobs
    (a Context, a raw handle, or None for the defaults)."""
    handle = getattr(ctx, "handle", ctx)
    return int(lib().dpc_job_footprint(handle, int(n), int(d), int(method)))


def dpc_probe_pair_rate(device: int, d: int, mode: int = 0):
    """(pairs/s, ms) of the register-resident pair test on every SM (mode 0
    direct 32-bit form, 1 direct 64-bit form, 2 expanded form for d <= 3)."""
    r, t = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib().dpc_probe_pair_rate(device, d, mode, ctypes.byref(r), ctypes.byref(t)), "dpc_probe_pair_rate")
    return r.value, t.value


def dpc_last_error() -> str:
    m = lib().dpc_last_error()
    return m.decode() if m else ""


def _check(status: int, where: str, ok=(DPC_OK,)) -> int:
    if status not in ok:
        raise DpcError(status, where, dpc_last_error())
    return status


# ---------------------------------------------------------------- raw calls

def dpc_create(device=0, stream_ptr=0, hbm_cap_bytes=0, mode=0, max_inflight=0, debug=0, tune_cache=None):
    o = DpcOptions(device, stream_ptr or None, hbm_cap_bytes, tune_cache.encode() if tune_cache else None, debug,
                   mode, max_inflight)
    h = ctypes.c_void_p()
    _check(lib().dpc_create(ctypes.byref(o), ctypes.byref(h)), "dpc_create")
    return h


def dpc_destroy(ctx):
    return _check(lib().dpc_destroy(ctx), "dpc_destroy")


def dpc_density(ctx, points_ptr, n, d, d_cut, is_device, rho_ptr=None):
    h = ctypes.c_void_p()
    _check(lib().dpc_density(ctx, points_ptr, n, d, d_cut, is_device, ctypes.byref(h), rho_ptr), "dpc_density")
    return h


def dpc_dependent(ds, dep_ptr=None, delta2_ptr=None):
    return _check(lib().dpc_dependent(ds, dep_ptr, delta2_ptr), "dpc_dependent")


def dpc_dependent_approx(ds, dep_ptr=None, delta2_ptr=None, exact_ptr=None):
    return _check(lib().dpc_dependent_approx(ds, dep_ptr, delta2_ptr, exact_ptr), "dpc_dependent_approx")


def dpc_sapprox(ctx, points_ptr, n, d, d_cut, eps_num, eps_den, is_device, rho_ptr=None, dep_ptr=None,
                delta2_ptr=None, pick_ptr=None):
    h = ctypes.c_void_p()
    _check(lib().dpc_sapprox(ctx, points_ptr, n, d, d_cut, int(eps_num), int(eps_den), is_device, ctypes.byref(h),
                             rho_ptr, dep_ptr, delta2_ptr, pick_ptr), "dpc_sapprox")
    return h


def dpc_cluster(ctx, points_ptr, n, d, d_cut, is_device, rho_min, delta_min, rho_ptr=None, dep_ptr=None,
                delta2_ptr=None, label_ptr=None) -> int:
    nc = ctypes.c_int64(0)
    _check(lib().dpc_cluster(ctx, points_ptr, n, d, int(d_cut), is_device, int(rho_min), int(delta_min), rho_ptr,
                             dep_ptr, delta2_ptr, label_ptr, ctypes.byref(nc)), "dpc_cluster")
    return int(nc.value)


def dpc_label(ds, rho_min, delta_min, label_ptr=None):
    nc = ctypes.c_int64(0)
    _check(lib().dpc_label(ds, int(rho_min), int(delta_min), label_ptr, ctypes.byref(nc)), "dpc_label")
    return int(nc.value)


def dpc_release(ds):
    return _check(lib().dpc_release(ds), "dpc_release")


def dpc_ds_info(ds) -> dict:
    info = DpcInfo()
    _check(lib().dpc_ds_info(ds, ctypes.byref(info)), "dpc_ds_info")
    return info.as_dict()


def dpc_autotune(ctx, jobs, repeats: int = 2) -> str:
    """Autotune on the sample jobs (a list of Job); returns the chosen setting."""
    arr = (DpcJob * len(jobs))(*[j.c for j in jobs])
    buf = ctypes.create_string_buffer(512)
    _check(lib().dpc_autotune(ctx, ctypes.cast(arr, ctypes.c_void_p), len(jobs), int(repeats), buf, 512),
           "dpc_autotune")
    return buf.value.decode()


def dpc_last_batch_info(ctx) -> dict:
    info = DpcInfo()
    _check(lib().dpc_last_batch_info(ctx, ctypes.byref(info)), "dpc_last_batch_info")
    return info.as_dict()


def dpc_set_profiling(ctx, on: bool):
    return _check(lib().dpc_set_profiling(ctx, 1 if on else 0), "dpc_set_profiling")


def dpc_set_tuning(ctx, key: str, value: int):
    return _check(lib().dpc_set_tuning(ctx, key.encode(), int(value)), "dpc_set_tuning")


def dpc_get_tuning(ctx, key: str) -> int:
    v = ctypes.c_int64(0)
    _check(lib().dpc_get_tuning(ctx, key.encode(), ctypes.byref(v)), "dpc_get_tuning")
    return int(v.value)


def dpc_submit(ctx, job: "DpcJob") -> int:
    t = ctypes.c_uint64(0)
    _check(lib().dpc_submit(ctx, ctypes.byref(job), ctypes.byref(t)), "dpc_submit")
    return int(t.value)


def dpc_poll(ctx, ticket: int):
    r = DpcResult()
    s = lib().dpc_poll(ctx, ticket, ctypes.byref(r))
    return s, r


def dpc_flush(ctx):
    return _check(lib().dpc_flush(ctx), "dpc_flush")


def dpc_wait(ctx, ticket: int, timeout_ms: int = -1):
    r = DpcResult()
    s = lib().dpc_wait(ctx, ticket, int(timeout_ms if timeout_ms >= 0 else 1 << 40), ctypes.byref(r))
    return s, r


# ---------------------------------------------------------------- wrappers

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _arg(x, dtype, shape=None):
    """(pointer, is_device) for a numpy array or a torch tensor."""
    if x is None:
        return None, 0
    if _is_torch(x):
        import torch
        want = {np.int32: torch.int32, np.int64: torch.int64, np.uint8: torch.uint8}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise ValueError(f"tensor must be contiguous {want}")
        if shape is not None and tuple(x.shape) != tuple(shape):
            raise ValueError(f"tensor shape {tuple(x.shape)} != {tuple(shape)}")
        return ctypes.c_void_p(x.data_ptr()), 1 if x.is_cuda else 0
    if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags.c_contiguous:
        raise ValueError(f"array must be a contiguous numpy {np.dtype(dtype).name} array")
    if shape is not None and x.shape != tuple(shape):
        raise ValueError(f"array shape {x.shape} != {tuple(shape)}")
    return x.ctypes.data_as(ctypes.c_void_p), 0


class Context:
    """A libdpc context on one device and one CUDA stream.

    With torch available the context runs on a torch CUDA stream
    (``self.stream``), so callers can time it with torch events and order
    their own work against it."""

    def __init__(self, device: int = 0, stream=None, mode: int = 0, hbm_cap_bytes: int = 0,
                 max_inflight: int = 0, debug: bool = False, profiling: bool = False, tune_cache=None):
        self.device = device
        self._kept = {}  # ticket -> Job submitted with keep
        self.stream = stream
        ptr = 0
        try:
            import torch
            if stream is None and torch.cuda.is_available():
                self.stream = torch.cuda.Stream(device=device)
            if self.stream is not None:
                ptr = self.stream.cuda_stream
        except ImportError:
            pass
        self.handle = dpc_create(device, ptr, hbm_cap_bytes, mode, max_inflight, 1 if debug else 0, tune_cache)
        if profiling:
            dpc_set_profiling(self.handle, True)

    def close(self):
        if self.handle is not None:
            dpc_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _order_after_torch(self, *tensors):
        if self.stream is None or not any(_is_torch(t) and t.is_cuda for t in tensors if t is not None):
            return
        import torch
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def density(self, points, d_cut: int, rho_out=None) -> "Dataset":
        if points.ndim != 2:
            raise ValueError("points must be n x d")
        n, d = int(points.shape[0]), int(points.shape[1])
        pp, dev = _arg(points, np.int32)
        rp, rdev = _arg(rho_out, np.int32, (n,))
        if rho_out is not None and rdev != dev:
            raise ValueError("rho_out must live where points live")
        self._order_after_torch(points, rho_out)
        h = dpc_density(self.handle, pp, n, d, int(d_cut), dev, rp)
        return Dataset(self, h, n, dev)

    def cluster(self, points, d_cut: int, rho_min: int, delta_min: int, rho_out=None, dep_out=None,
                delta2_out=None, label_out=None) -> int:
        """The whole path in one call (dpc_cluster); returns the number of
        centers. Outputs live where the points live."""
        if points.ndim != 2:
            raise ValueError("points must be n x d")
        n, d = int(points.shape[0]), int(points.shape[1])
        pp, dev = _arg(points, np.int32)
        ptrs = []
        for x, dt in [(rho_out, np.int32), (dep_out, np.int32), (delta2_out, np.int64), (label_out, np.int32)]:
            p, xdev = _arg(x, dt, (n,))
            if x is not None and xdev != dev:
                raise ValueError("outputs must live where points live")
            ptrs.append(p)
        self._order_after_torch(points, rho_out, dep_out, delta2_out, label_out)
        return dpc_cluster(self.handle, pp, n, d, int(d_cut), dev, rho_min, delta_min, *ptrs)

    def sapprox(self, points, d_cut: int, eps, rho_out=None, dep_out=None, delta2_out=None,
                pick_out=None) -> "Dataset":
        """S-Approx-DPC (Section 5) with eps = (num, den), or a float read as
        num / 10^6; labels of the returned dataset follow its picks."""
        if points.ndim != 2:
            raise ValueError("points must be n x d")
        num, den = eps_fraction(eps)
        n, d = int(points.shape[0]), int(points.shape[1])
        pp, dev = _arg(points, np.int32)
        outs = [(rho_out, np.int32), (dep_out, np.int32), (delta2_out, np.int64), (pick_out, np.uint8)]
        ptrs = []
        for x, dt in outs:
            p, xdev = _arg(x, dt, (n,))
            if x is not None and xdev != dev:
                raise ValueError("outputs must live where points live")
            ptrs.append(p)
        self._order_after_torch(points, rho_out, dep_out, delta2_out, pick_out)
        h = dpc_sapprox(self.handle, pp, n, d, int(d_cut), num, den, dev, *ptrs)
        return Dataset(self, h, n, dev)

    def tune(self, **knobs):
        """Set tuning knobs (speed only; results are unchanged)."""
        for k, val in knobs.items():
            dpc_set_tuning(self.handle, k, val)

    def tuning(self, key: str) -> int:
        return dpc_get_tuning(self.handle, key)

    def submit(self, job: "Job") -> int:
        t = dpc_submit(self.handle, job.c)
        job.ticket = t
        if job.c.keep:
            self._kept[t] = job
        return t

    def flush(self):
        return dpc_flush(self.handle)

    def _adopt(self, ticket: int, s: int, r):
        """A job submitted with keep: its device state becomes job.dataset."""
        job = self._kept.pop(ticket, None) if s != DPC_PENDING else None
        if job is not None and r.dataset:
            job.dataset = Dataset(self, ctypes.c_void_p(r.dataset), job.n, job.is_device)
        return s, r

    def poll(self, ticket: int):
        return self._adopt(ticket, *dpc_poll(self.handle, ticket))

    def wait(self, ticket: int, timeout_ms: int = -1):
        return self._adopt(ticket, *dpc_wait(self.handle, ticket, timeout_ms))

    def last_batch_info(self) -> dict:
        return dpc_last_batch_info(self.handle)

    def autotune(self, jobs, repeats: int = 2) -> str:
        return dpc_autotune(self.handle, jobs, repeats)


class Dataset:
    """A dataset clustered on the device (rho done; dep/labels on demand)."""

    def __init__(self, ctx: Context, handle, n: int, is_device: int):
        self.ctx, self.handle, self.n, self.is_device = ctx, handle, n, is_device

    def _out(self, x, dtype, shape):
        p, dev = _arg(x, dtype, shape)
        if x is not None and dev != self.is_device:
            raise ValueError("outputs must live where the dataset's input lived")
        return p

    def dependent(self, dep_out=None, delta2_out=None):
        self.ctx._order_after_torch(dep_out, delta2_out)
        dpc_dependent(self.handle, self._out(dep_out, np.int32, (self.n,)),
                      self._out(delta2_out, np.int64, (self.n,)))

    def dependent_approx(self, dep_out=None, delta2_out=None, exact_out=None):
        """Approx-DPC's dependent points (Section 4.3); later labels use them."""
        self.ctx._order_after_torch(dep_out, delta2_out, exact_out)
        dpc_dependent_approx(self.handle, self._out(dep_out, np.int32, (self.n,)),
                             self._out(delta2_out, np.int64, (self.n,)), self._out(exact_out, np.uint8, (self.n,)))

    def label(self, rho_min: int, delta_min: int, label_out=None) -> int:
        self.ctx._order_after_torch(label_out)
        return dpc_label(self.handle, rho_min, delta_min, self._out(label_out, np.int32, (self.n,)))

    def info(self) -> dict:
        return dpc_ds_info(self.handle)

    def release(self):
        if self.handle is not None:
            dpc_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Job:
    """One dataset + (rho_min, delta_min) queries for dpc_submit, with output
    arrays allocated here (rho, dep, delta2, labels[q], n_centers[q], and
    aux: Approx-DPC's exact flags or S-Approx-DPC's picks). Host numpy points
    give host outputs; a CUDA tensor of points gives device outputs (torch
    tensors on its device) and a device-memory job. method: "exact",
    "approx" or "sapprox" (with eps as for Context.sapprox)."""

    def __init__(self, points, d_cut: int, queries, method: str = "exact", eps=(4, 5), keep: bool = False,
                 pinned: bool = False):
        q = list(queries)
        self.rho_min = np.array([int(a) for a, _ in q], dtype=np.int64)
        self.delta_min = np.array([int(b) for _, b in q], dtype=np.int64)
        self.n_centers = np.empty(len(q), np.int64)
        if _is_torch(points) and points.is_cuda:
            import torch
            if points.dtype != torch.int32 or not points.is_contiguous() or points.ndim != 2:
                raise ValueError("device points must be a contiguous n x d int32 tensor")
            self.points = points
            n, d = int(points.shape[0]), int(points.shape[1])
            dev = points.device
            self.rho = torch.empty(n, dtype=torch.int32, device=dev)
            self.dep = torch.empty(n, dtype=torch.int32, device=dev)
            self.delta2 = torch.empty(n, dtype=torch.int64, device=dev)
            self.label = torch.empty((len(q), n), dtype=torch.int32, device=dev)
            self.aux = torch.empty(n, dtype=torch.uint8, device=dev)
            p = lambda a: ctypes.c_void_p(a.data_ptr() if a.numel() else 0)
            is_dev = 1
        else:
            self.points = np.ascontiguousarray(points, dtype=np.int32)
            n, d = self.points.shape
            if pinned:
                # page-locked host outputs: in a batch the device writes them
                # directly (one pass for all such jobs) instead of one copy each
                import torch
                e = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
                self.rho, self.dep = e(n, torch.int32), e(n, torch.int32)
                self.delta2, self.label = e(n, torch.int64), e((len(q), n), torch.int32)
                self.aux = e(n, torch.uint8)
            else:
                self.rho = np.empty(n, np.int32)
                self.dep = np.empty(n, np.int32)
                self.delta2 = np.empty(n, np.int64)
                self.label = np.empty((len(q), n), np.int32)
                self.aux = np.empty(n, np.uint8)
            p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
            is_dev = 0
        h = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        if method not in METHODS:
            raise ValueError(f"method must be one of {sorted(METHODS)}")
        self.method = method
        num, den = eps_fraction(eps)
        self.c = DpcJob(p(self.points), n, d, int(d_cut), len(q), h(self.rho_min), h(self.delta_min),
                        p(self.rho), p(self.dep), p(self.delta2), p(self.label), h(self.n_centers), is_dev,
                        METHODS[method], num, den, p(self.aux))
        self.c.keep = 1 if keep else 0
        self.n, self.is_device = n, is_dev
        self.dataset = None  # keep: the finished job's device state (Dataset), for re-queries
        self.ticket = None


def eps_fraction(eps):
    """(num, den) of S-Approx-DPC's eps: a pair as given, or a float rounded
    to a multiple of 10^-6 and reduced."""
    import math
    if isinstance(eps, tuple):
        num, den = int(eps[0]), int(eps[1])
    else:
        num, den = int(round(float(eps) * 10 ** 6)), 10 ** 6
        g = math.gcd(num, den)
        num, den = num // g, den // g
    if num < 1 or den < 1:
        raise ValueError("eps must be positive")
    return num, den


def cluster_sapprox(points: np.ndarray, d_cut: int, eps, rho_min: int, delta_min: int, device: int = 0) -> dict:
    """S-Approx-DPC on host arrays: rho (-1 where not picked), dep, delta2,
    pick, label, n_centers."""
    pts = np.ascontiguousarray(points, dtype=np.int32)
    n = pts.shape[0]
    with Context(device) as ctx:
        rho = np.empty(n, np.int32)
        dep = np.empty(n, np.int32)
        d2 = np.empty(n, np.int64)
        pk = np.empty(n, np.uint8)
        ds = ctx.sapprox(pts, d_cut, eps, rho, dep, d2, pk)
        lab = np.empty(n, np.int32)
        nc = ds.label(rho_min, delta_min, lab)
        ds.release()
    return {"rho": rho, "dep": dep, "delta2": d2, "pick": pk.astype(bool), "label": lab, "n_centers": nc}


def cluster_approx(points: np.ndarray, d_cut: int, rho_min: int, delta_min: int, device: int = 0) -> dict:
    """Approx-DPC on host arrays: rho, dep, delta2, exact, label, n_centers."""
    pts = np.ascontiguousarray(points, dtype=np.int32)
    n = pts.shape[0]
    with Context(device) as ctx:
        rho = np.empty(n, np.int32)
        ds = ctx.density(pts, d_cut, rho)
        dep = np.empty(n, np.int32)
        d2 = np.empty(n, np.int64)
        ex = np.empty(n, np.uint8)
        ds.dependent_approx(dep, d2, ex)
        lab = np.empty(n, np.int32)
        nc = ds.label(rho_min, delta_min, lab)
        ds.release()
    return {"rho": rho, "dep": dep, "delta2": d2, "exact": ex.astype(bool), "label": lab, "n_centers": nc}


def cluster(points: np.ndarray, d_cut: int, rho_min: int, delta_min: int, device: int = 0) -> dict:
    """The whole path on host arrays (dpc_cluster): rho, dep, delta2, label,
    n_centers."""
    pts = np.ascontiguousarray(points, dtype=np.int32)
    n = pts.shape[0]
    with Context(device) as ctx:
        rho = np.empty(n, np.int32)
        dep = np.empty(n, np.int32)
        d2 = np.empty(n, np.int64)
        lab = np.empty(n, np.int32)
        nc = ctx.cluster(pts, d_cut, rho_min, delta_min, rho, dep, d2, lab)
    return {"rho": rho, "dep": dep, "delta2": d2, "label": lab, "n_centers": nc}
