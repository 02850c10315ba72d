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


def _call(L, dpc, torch, rho, dep, d2, rmin, dmin, n=None):
    n = len(rho) if n is None else n
    r = torch.tensor(rho, dtype=torch.int32, device="cuda")
    q = torch.tensor(dep, dtype=torch.int32, device="cuda")
    e = torch.tensor(d2, dtype=torch.int64, device="cuda")
    lab = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    nc = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    s = L.dpc_label_static(_p(r), _p(q), _p(e), n, rmin, dmin, _p(lab), _p(nc), None)
    torch.cuda.synchronize()
    return s, lab[:n].cpu().tolist(), int(nc.item())


BIG = (1 << 63) - 1
# six points: 0 is the densest, 5 is noise for rho_min 2, the rest hang on
# their links (delta2 1 is below delta_min^2)
RHO = [9, 8, 8, 7, 7, 1]
D2 = [BIG, 1, 1, 1, 1, 1]


def test_static_labels_follow_valid_links(env):
    dpc, L, torch = env
    s, lab, nc = _call(L, dpc, torch, RHO, [-1, 0, 1, 0, 3, 4], D2, 2, 5)
    assert s == dpc.DPC_OK
    assert lab == [0, 0, 0, 0, 0, -1] and nc == 1


@pytest.mark.parametrize("bad,rejected", [
    ({3: 4}, [3, 4]),            # 3 -> 4 -> 3: equal density, 4 is not higher than 3 (a 2-cycle)
    ({1: 1 << 23}, [1, 2]),      # far outside the arrays: never read
    ({1: 6}, [1, 2]),            # just past the end
    ({2: -3}, [2]),              # negative
    ({4: 4}, [4]),               # a point hanging on itself without being a center
    ({1: 3}, [1, 2]),            # a lower point
])
def test_static_labels_reject_links_that_are_not_a_forest(env, bad, rejected):
    dpc, L, torch = env
    dep = [-1, 0, 1, 0, 3, 4]
    for i, q in bad.items():
        dep[i] = q
    s, lab, nc = _call(L, dpc, torch, RHO, dep, D2, 2, 5)
    assert s == dpc.DPC_OK  # the call only queues the work
    want = [0, 0, 0, 0, 0, -1]
    for i in rejected:
        want[i] = -2
    assert lab == want
    assert nc == -1
    # the next call starts from a clear error word
    s, lab, nc = _call(L, dpc, torch, RHO, [-1, 0, 1, 0, 3, 4], D2, 2, 5)
    assert lab == [0, 0, 0, 0, 0, -1] and nc == 1


def test_static_labels_empty_and_parameter_bounds(env):
    dpc, L, torch = env
    s, lab, nc = _call(L, dpc, torch, [1], [-1], [BIG], 1, 5, n=0)
    assert s == dpc.DPC_OK and lab == [] and nc == 0
    for dmin in (0, -1, 3037000500):
        s, _, _ = _call(L, dpc, torch, RHO, [-1, 0, 1, 0, 3, 4], D2, 2, dmin)
        assert s == dpc.DPC_ERR_INVALID_ARG
    for dmin in (1, 3037000499):
        s, lab, nc = _call(L, dpc, torch, RHO, [-1, 0, 1, 0, 3, 4], D2, 2, dmin)
        assert s == dpc.DPC_OK
        # delta_min 1: every non-noise point is a center (delta2 1 >= 1)
        assert nc == (5 if dmin == 1 else 1)


def test_static_labels_allocate_nothing(env):
    dpc, L, torch = env
    ds = workloads.random_blobs(506, 20000, 2, 2000, blobs=5, spread=0.05, dup=3)
    n = ds.n
    pts = torch.from_numpy(ds.points).cuda()
    rho = torch.empty(n, dtype=torch.int32, device="cuda")
    dep = torch.empty(n, dtype=torch.int32, device="cuda")
    d2 = torch.empty(n, dtype=torch.int64, device="cuda")
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    nc = torch.empty(1, dtype=torch.int64, device="cuda")
    with dpc.Context(0) as ctx:
        h = ctx.density(pts, ds.d_cut, rho)
        h.dependent(dep, d2)
        h.release()
    args = (_p(rho), _p(dep), _p(d2), n, ds.rho_min, ds.delta_min, _p(lab), _p(nc), None)
    assert L.dpc_label_static(*args) == dpc.DPC_OK  # first call on the device: the set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert L.dpc_label_static(*args) == dpc.DPC_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert int(nc.item()) >= 1
