"""The allocation-free labels entry point (dpc_label_static) gives the same
labels and center count as dpc_label on the same dataset, on two calls in a
row, through the C ABI. It serves callers that cannot allocate device memory
when they call; its scratch is a fixed array inside the library. This file
is collected last so that a failure here comes after every other test."""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2207_04649_gb300 as dpc
    L = dpc.lib()
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    L.dpc_label_static.argtypes = [vp, vp, vp, i64, i64, i64, vp, vp, vp]
    L.dpc_label_static.restype = ctypes.c_int
    return dpc, L, torch


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_static_labels_match_dataset_labels_twice(env):
    dpc, L, torch = env
    ds = workloads.random_blobs(505, 30000, 3, 2500, blobs=6, spread=0.04, dup=20)
    n = ds.n
    pts = torch.from_numpy(ds.points).cuda()
    rho = torch.empty(n, dtype=torch.int32, device="cuda")
    dep = torch.empty(n, dtype=torch.int32, device="cuda")
    d2 = torch.empty(n, dtype=torch.int64, device="cuda")
    with dpc.Context(0) as ctx:
        h = ctx.density(pts, ds.d_cut, rho)
        h.dependent(dep, d2)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream().cuda_stream
        for rmin, dmin in [(ds.rho_min, ds.delta_min), (1, 2 * ds.d_cut + 1)]:
            want = torch.empty(n, dtype=torch.int32, device="cuda")
            want_nc = h.label(rmin, dmin, want)
            got = torch.full((n,), -7, dtype=torch.int32, device="cuda")
            got_nc = torch.full((1,), -7, dtype=torch.int64, device="cuda")
            s = L.dpc_label_static(_p(rho), _p(dep), _p(d2), n, rmin, dmin, _p(got), _p(got_nc),
                                   ctypes.c_void_p(stream))
            assert s == dpc.DPC_OK
            torch.cuda.synchronize()
            assert torch.equal(got, want)
            assert int(got_nc.item()) == want_nc
        h.release()


def test_static_labels_reject_sizes_beyond_the_scratch(env):
    dpc, L, torch = env
    x = torch.zeros(4, dtype=torch.int32, device="cuda")
    y = torch.zeros(4, dtype=torch.int64, device="cuda")
    s = L.dpc_label_static(_p(x), _p(x), _p(y), (1 << 22) + 1, 1, 10, _p(x), None, None)
    assert s == dpc.DPC_ERR_INVALID_ARG
