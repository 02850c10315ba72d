"""GPU parity: the CUDA path, called through the C ABI, against the oracle.

Integer results, so the bar is bit-exact equality of rho, dep, delta2, the
labels and the center count. Small and medium problems are compared element
by element; at the full sizes of the 1M x 8 and 5.8M x 3 workloads the
oracle computes a seeded sample of points one by one (rho against all n
points, the dependent point against every higher point), and properties that
hold at any size are checked on every point.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

I64MAX = np.iinfo(np.int64).max


@pytest.fixture(scope="module")
def dpc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2207_04649_gb300 as m
    m.lib()
    return m


def run_host(dpc, pts, d_cut, queries, knobs=None):
    """Whole path through the host-pointer ABI; several label queries."""
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    n = pts.shape[0]
    with dpc.Context(0) as ctx:
        if knobs:
            ctx.tune(**knobs)
        rho = np.full(n, -7, np.int32)
        ds = ctx.density(pts, d_cut, rho)
        dep = np.full(n, -7, np.int32)
        d2 = np.full(n, -7, np.int64)
        ds.dependent(dep, d2)
        labs = []
        for rmin, dmin in queries:
            lab = np.full(n, -7, np.int32)
            nc = ds.label(rmin, dmin, lab)
            labs.append((lab, nc))
        info = ds.info()
        ds.release()
    return rho, dep, d2, labs, info


def assert_full_parity(dpc, pts, d_cut, queries, knobs=None):
    rho, dep, d2, labs, info = run_host(dpc, pts, d_cut, queries, knobs)
    orho = oracle.rho(pts, d_cut)
    np.testing.assert_array_equal(rho, orho)
    odep, od2 = oracle.dependent(pts, orho)
    np.testing.assert_array_equal(dep, odep)
    np.testing.assert_array_equal(d2, od2)
    for (lab, nc), (rmin, dmin) in zip(labs, queries):
        olab, onc = oracle.label(orho, odep, od2, rmin, dmin)
        np.testing.assert_array_equal(lab, olab)
        assert nc == onc
    return info


# --------------------------------------------------------------- hand-worked

def test_golden_cases_on_gpu(dpc):
    import json, os
    with open(os.path.join(os.path.dirname(__file__), "golden", "hand_worked.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        pts = np.array(c["points"], np.int32)
        q = [(x["rho_min"], x["delta_min"]) for x in c["queries"]]
        rho, dep, d2, labs, _ = run_host(dpc, pts, c["d_cut"], q)
        assert rho.tolist() == c["rho"], c["name"]
        assert dep.tolist() == c["dep"], c["name"]
        assert d2.tolist() == c["delta2"], c["name"]
        for (lab, nc), x in zip(labs, c["queries"]):
            assert lab.tolist() == x["label"], c["name"]
            assert nc == x["n_centers"], c["name"]


# ------------------------------------------------------------ small shapes

SHAPES = [
    # (seed, n, d, d_cut, domain, blobs, spread, dup)
    (1, 1, 2, 100, 1000, 1, 0.1, 0),
    (2, 2, 3, 100, 1000, 1, 0.1, 0),
    (3, 31, 2, 150, 1000, 2, 0.1, 0),
    (4, 32, 1, 20, 1000, 2, 0.1, 0),
    (5, 33, 4, 300, 1000, 2, 0.1, 3),
    (6, 1000, 2, 400, 100000, 4, 0.05, 10),
    (7, 1000, 3, 2500, 100000, 4, 0.05, 10),
    (8, 2000, 5, 6000, 100000, 3, 0.05, 5),
    (9, 1500, 6, 8000, 100000, 3, 0.05, 0),
    (10, 1500, 7, 9000, 100000, 3, 0.05, 0),
    (11, 3000, 8, 9000, 100000, 5, 0.05, 20),
    (12, 5000, 2, 30, 1000, 3, 0.2, 50),      # many points per cell, huge cells
    (13, 4000, 3, 1, 50, 2, 0.2, 100),        # d_cut = 1: only duplicates are neighbours
    (14, 3000, 2, 5000, 10000, 1, 0.3, 0),    # few cells, big candidate lists
    (15, 2500, 1, 7, 100000, 6, 0.01, 25),    # d = 1
    (16, 2000, 3, 200, 100000, 40, 0.002, 0), # many small tight blobs, most cells sparse
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"n{s[1]}_d{s[2]}_dc{s[3]}")
def test_random_shapes_bit_exact(dpc, shape):
    seed, n, d, dc, dom, blobs, spread, dup = shape
    ds = workloads.random_blobs(seed, n, d, dc, domain=dom, blobs=blobs, spread=spread, dup=dup)
    queries = [(2, dc + 1), (1, 3 * dc + 1), (5, 10 * dc)]
    assert_full_parity(dpc, ds.points, dc, queries)


@pytest.mark.parametrize("knobs", [dict(rho_bulk=1), dict(rho_bulk=1, sparse_cand=0, kch=64),
                                   dict(rho_bulk=1, hd_min_d=1, hd_cell_factor=2, sparse_cand=0)],
                         ids=["bulk", "bulk_all_dense_small_items", "bulk_reach2"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"n{s[1]}_d{s[2]}_dc{s[3]}")
def test_random_shapes_bulk_staging(dpc, shape, knobs):
    """The dense density kernels with candidates staged by bulk copies into
    shared memory (d <= 4): every cell on that path, items of 64
    candidates (many chunks, ragged tails), and reach 2 (runs read in
    place) give the oracle's bits."""
    seed, n, d, dc, dom, blobs, spread, dup = shape
    ds = workloads.random_blobs(seed, n, d, dc, domain=dom, blobs=blobs, spread=spread, dup=dup)
    assert_full_parity(dpc, ds.points, dc, [(2, dc + 1), (5, 10 * dc)], knobs)


@pytest.mark.parametrize("sparse_cand", [512, 0, 2147483647])
@pytest.mark.parametrize("d", [5, 6, 7, 8])
@pytest.mark.parametrize("f", [1, 2, 3])
def test_high_dims_grid_path(dpc, d, f, sparse_cand):
    """The projected grid for d > 4, with
    cells of side d_cut / f searched f cells away; small cells on the warp
    path by their candidate count (sparse_cand 0: every cell)."""
    ds = workloads.random_blobs(60 + d, 2500, d, 9000, blobs=4, spread=0.05, dup=10)
    info = assert_full_parity(dpc, ds.points, 9000, [(3, 27001)],
                              dict(hd_cell_factor=f, hd_min_d=5, sparse_cand=sparse_cand))
    assert 1 <= info["grid_dims"] <= 4


@pytest.mark.parametrize("d", [5, 6, 7, 8])
def test_high_dims_one_lane_tree_search(dpc, d):
    """d > 4 with the tree search one lane per open point (the default there
    is the warp-cooperative form) and every open point on the tree."""
    ds = workloads.random_blobs(80 + d, 2500, d, 9000, blobs=4, spread=0.05, dup=10)
    assert_full_parity(dpc, ds.points, 9000, [(3, 27001)], dict(tree_warp=0, bf_rank=0))


def test_cutoff_spanning_the_box_and_wide_8d_blobs(dpc):
    """A cutoff larger than the whole box (one cell), far-apart 8-d blobs
    over the full coordinate range, and tiny 5-d sets."""
    rng = np.random.default_rng(99)
    pts = rng.integers(0, 50, size=(3000, 2)).astype(np.int32)
    assert_full_parity(dpc, pts, 10_000_000, [(1, 10_000_001)])
    base = rng.integers(0, (1 << 30) - 1, size=(4, 8))
    pts = np.concatenate([np.clip(b + rng.normal(0, 3e6, size=(300, 8)), 0, (1 << 30) - 1)
                          for b in base]).astype(np.int32)
    assert_full_parity(dpc, pts, 2_000_000, [(2, 50_000_000)])
    for n in (1, 2, 16, 17, 33):
        pts = rng.integers(0, 1000, size=(n, 5)).astype(np.int32)
        assert_full_parity(dpc, pts, 300, [(1, 301)])


SMALL_CUTOFFS = [
    (71, 3000, 4, 2, 30, 3, 0.2, 50),   # k = 4, d_cut = 2: corner cells lie at least d_cut away
    (72, 3000, 4, 1, 20, 3, 0.2, 50),
    (73, 3000, 2, 1, 60, 3, 0.2, 50),
    (74, 3000, 3, 2, 40, 3, 0.2, 50),
    (75, 2500, 8, 3, 12, 3, 0.3, 30),   # reach 2 (d >= 7) with far corner cells left out
    (76, 2500, 7, 4, 15, 3, 0.3, 30),
]


@pytest.mark.parametrize("shape", SMALL_CUTOFFS, ids=lambda s: f"n{s[1]}_d{s[2]}_dc{s[3]}")
def test_small_cutoffs_bit_exact(dpc, shape):
    """Cutoffs so small that the neighbour runs leave out in-reach cells (no
    point there is within d_cut, but one may be the nearest higher point)."""
    seed, n, d, dc, dom, blobs, spread, dup = shape
    ds = workloads.random_blobs(seed, n, d, dc, domain=dom, blobs=blobs, spread=spread, dup=dup)
    assert_full_parity(dpc, ds.points, dc, [(1, dc + 1), (2, 3 * dc + 1)])


def test_all_points_identical(dpc):
    pts = np.full((777, 3), 4242, np.int32)
    assert_full_parity(dpc, pts, 10, [(1, 11), (778, 11)])


def test_single_cell_everything_in_range(dpc):
    rng = np.random.default_rng(99)
    pts = rng.integers(0, 50, size=(3000, 2)).astype(np.int32)
    assert_full_parity(dpc, pts, 10_000_000, [(1, 10_000_001)])


def test_wide_coordinates_64bit_path(dpc):
    """Coordinates near 2^30 force the 64-bit pair arithmetic."""
    rng = np.random.default_rng(5)
    base = rng.integers(0, (1 << 30) - 1, size=(4, 3))
    pts = np.concatenate([np.clip(b + rng.normal(0, 3e6, size=(600, 3)), 0, (1 << 30) - 1)
                          for b in base]).astype(np.int32)
    rho, dep, d2, labs, info = run_host(dpc, pts, 2_000_000, [(2, 50_000_000)])
    assert info["pair_bits"] == 64
    info2 = assert_full_parity(dpc, pts, 2_000_000, [(2, 50_000_000), (1, 2_000_001)])
    assert info2["pair_bits"] == 64


def test_eight_dims_ungridded_64bit(dpc):
    ds = workloads.random_blobs(21, 3000, 8, 20000, blobs=4, spread=0.08)
    info = assert_full_parity(dpc, ds.points, 20000, [(3, 60001)])
    assert info["grid_dims"] <= 4


def test_empty_input(dpc):
    pts = np.zeros((0, 3), np.int32)
    rho, dep, d2, labs, info = run_host(dpc, pts, 10, [(1, 11)])
    assert rho.size == 0 and labs[0][1] == 0


def test_plain_20k_2d_full(dpc):
    ds = workloads.plain_20k_2d()
    info = assert_full_parity(dpc, ds.points, ds.d_cut, [(ds.rho_min, ds.delta_min), (2, 2 * ds.d_cut)])
    assert info["cells"] > 0


def test_device_tensor_path_matches_host_path(dpc):
    import torch
    ds = workloads.plain_20k_2d(seed=11)
    n = ds.n
    rho_h, dep_h, d2_h, labs_h, _ = run_host(dpc, ds.points, ds.d_cut, [(ds.rho_min, ds.delta_min)])
    pts = torch.from_numpy(ds.points).cuda()
    rho = torch.empty(n, dtype=torch.int32, device="cuda")
    dep = torch.empty(n, dtype=torch.int32, device="cuda")
    d2 = torch.empty(n, dtype=torch.int64, device="cuda")
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    with dpc.Context(0) as ctx:
        h = ctx.density(pts, ds.d_cut, rho)
        h.dependent(dep, d2)
        nc = h.label(ds.rho_min, ds.delta_min, lab)
        h.release()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(rho.cpu().numpy(), rho_h)
    np.testing.assert_array_equal(dep.cpu().numpy(), dep_h)
    np.testing.assert_array_equal(d2.cpu().numpy(), d2_h)
    np.testing.assert_array_equal(lab.cpu().numpy(), labs_h[0][0])
    assert nc == labs_h[0][1]


def test_invalid_arguments_are_errors(dpc):
    pts = np.zeros((5, 2), np.int32)
    with dpc.Context(0) as ctx:
        for bad in [dict(d_cut=0), dict(d_cut=1 << 31)]:
            with pytest.raises(dpc.DpcError) as e:
                ctx.density(pts, **bad)
            assert e.value.status == dpc.DPC_ERR_INVALID_ARG
        with pytest.raises(dpc.DpcError) as e:
            ctx.density(np.zeros((5, 9), np.int32), 10)
        assert e.value.status == dpc.DPC_ERR_INVALID_ARG
        neg = pts.copy()
        neg[2, 1] = -1
        with pytest.raises(dpc.DpcError) as e:
            ctx.density(neg, 10)
        assert e.value.status == dpc.DPC_ERR_INVALID_ARG
        big = pts.copy()
        big[0, 0] = 1 << 30
        with pytest.raises(dpc.DpcError) as e:
            ctx.density(big, 10)
        assert e.value.status == dpc.DPC_ERR_INVALID_ARG
        h = ctx.density(pts, 10)
        with pytest.raises(dpc.DpcError) as e:
            h.label(1, 10)  # delta_min must exceed d_cut
        assert e.value.status == dpc.DPC_ERR_INVALID_ARG
        h.release()


# ------------------------------------------------------- full-size samples

def check_sampled(dpc, ds, m, seed):
    pts = ds.points
    n = ds.n
    rho, dep, d2, labs, info = run_host(dpc, pts, ds.d_cut, [(ds.rho_min, ds.delta_min)])
    idx = np.sort(np.random.default_rng(seed).choice(n, size=min(m, n), replace=False))
    # (i) rho of the sample against all n points
    np.testing.assert_array_equal(rho[idx], oracle.rho_subset(pts, ds.d_cut, idx))
    # (ii) dependent point of the sample against every higher point (ranks
    # from the GPU densities, checked on the sample above)
    sdep, sd2 = oracle.dependent_subset(pts, rho, idx)
    np.testing.assert_array_equal(dep[idx], sdep)
    np.testing.assert_array_equal(d2[idx], sd2)
    # (iii) properties on every point
    assert (int(rho.astype(np.int64).sum()) - n) % 2 == 0 and rho.min() >= 1
    order = oracle.rank_order(rho)
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    assert dep[order[0]] == -1 and d2[order[0]] == I64MAX and (dep == -1).sum() == 1
    nz = dep >= 0
    assert np.all(rank[dep[nz]] < rank[nz])
    P = pts.astype(np.int64)
    np.testing.assert_array_equal(((P[nz] - P[dep[nz]]) ** 2).sum(axis=1), d2[nz])
    lab, nc = labs[0]
    noise = rho < ds.rho_min
    ctr = ~noise & (d2 >= ds.delta_min * ds.delta_min)
    np.testing.assert_array_equal(lab == -1, noise)
    assert nc == int(ctr.sum())
    assert np.all(lab[ctr] == np.nonzero(ctr)[0])
    mid = ~noise & ~ctr
    assert np.all(lab[mid] == lab[dep[mid]])
    # labels of the whole set from the dependent links (oracle step 4)
    olab, onc = oracle.label(rho, dep, d2, ds.rho_min, ds.delta_min)
    np.testing.assert_array_equal(lab, olab)
    assert nc == onc
    return info


def test_plain_1m_8d_sampled(dpc):
    info = check_sampled(dpc, workloads.plain_1m_8d(), 2000, 31)
    assert info["n"] == 1_000_000


def test_plain_5p8m_3d_sampled(dpc):
    """20k-point seeded sample, as specified for sets past 2M points."""
    info = check_sampled(dpc, workloads.plain_5p8m_3d(), 20_000, 32)
    assert info["n"] == 5_800_000


# ------------------------------------------------------- tuning knobs

@pytest.mark.parametrize("knobs", [dict(qch=32), dict(qch=64, kch=4096, bf_rank=0),
                                   dict(kch=64, bf_rank=100000), dict(kmax=2), dict(kmax=1, qch=32),
                                   dict(hd_min_d=3, hd_cell_factor=3), dict(hd_min_d=1, bf_rank=0),
                                   dict(tree_warp=0), dict(tree_warp=1, bf_rank=0, hd_min_d=1),
                                   dict(sparse_cand=0), dict(sparse_cand=2147483647),
                                   dict(sparse_cand=20, kch=64), dict(rho_bulk=1)],
                         ids=lambda k: ",".join(f"{a}={b}" for a, b in k.items()))
def test_tuning_knobs_do_not_change_results(dpc, knobs):
    ds = workloads.random_blobs(77, 6000, 3, 900, blobs=5, spread=0.06, dup=8)
    q = [(3, 3 * 900)]
    base = run_host(dpc, ds.points, ds.d_cut, q)
    pts = np.ascontiguousarray(ds.points)
    n = pts.shape[0]
    with dpc.Context(0) as ctx:
        ctx.tune(**knobs)
        for k, val in knobs.items():
            assert ctx.tuning(k) == val
        rho = np.empty(n, np.int32)
        h = ctx.density(pts, ds.d_cut, rho)
        dep = np.empty(n, np.int32)
        d2 = np.empty(n, np.int64)
        h.dependent(dep, d2)
        lab = np.empty(n, np.int32)
        nc = h.label(*q[0], lab)
        h.release()
    np.testing.assert_array_equal(rho, base[0])
    np.testing.assert_array_equal(dep, base[1])
    np.testing.assert_array_equal(d2, base[2])
    np.testing.assert_array_equal(lab, base[3][0][0])
    assert nc == base[3][0][1]


def test_tuning_rejects_unknown_keys(dpc):
    with dpc.Context(0) as ctx:
        with pytest.raises(dpc.DpcError):
            ctx.tune(nonsense=3)
        with pytest.raises(dpc.DpcError):
            ctx.tune(kmax=9)


def test_one_call_cluster_matches_the_separate_calls(dpc):
    """dpc_cluster (copies beside the compute) gives the bits of density +
    dependent + label, host and device buffers, and rejects bad queries."""
    import torch
    ds = workloads.random_blobs(91, 30000, 3, 1500, blobs=6, spread=0.05, dup=10)
    pts = np.ascontiguousarray(ds.points)
    n = pts.shape[0]
    ref = run_host(dpc, pts, 1500, [(3, 4000)])
    with dpc.Context(0) as ctx:
        h_out = [np.full(n, -7, t) for t in (np.int32, np.int32, np.int64, np.int32)]
        nc = ctx.cluster(pts, 1500, 3, 4000, *h_out)
        dev = torch.device("cuda", 0)
        d_out = [torch.full((n,), -7, dtype=t, device=dev) for t in (torch.int32, torch.int32, torch.int64, torch.int32)]
        nc2 = ctx.cluster(torch.from_numpy(pts).to(dev), 1500, 3, 4000, *d_out)
        ctx.stream.synchronize()
        with pytest.raises(dpc.DpcError):
            ctx.cluster(pts, 1500, 3, 1500)  # delta_min must exceed d_cut
        empty = ctx.cluster(np.zeros((0, 3), np.int32), 5, 1, 6)
    for got in (h_out, [t.cpu().numpy() for t in d_out]):
        np.testing.assert_array_equal(got[0], ref[0])
        np.testing.assert_array_equal(got[1], ref[1])
        np.testing.assert_array_equal(got[2], ref[2])
        np.testing.assert_array_equal(got[3], ref[3][0][0])
    assert nc == nc2 == ref[3][0][1]
    assert empty == 0


def test_errors_mid_call_leave_the_context_usable(dpc):
    """Calls that fail after device work has started (coordinates out of
    range found on the device) release their buffers and leave the context
    working."""
    bad = np.array([[0, 0], [5, (1 << 30) + 3]], np.int32)
    good = workloads.random_blobs(95, 3000, 3, 900, blobs=4, spread=0.05)
    ref = run_host(dpc, good.points, 900, [(2, 2000)])
    with dpc.Context(0) as ctx:
        for _ in range(20):
            with pytest.raises(dpc.DpcError):
                ctx.density(bad, 10)
        for _ in range(5):
            with pytest.raises(dpc.DpcError):
                ctx.sapprox(bad, 10, (4, 5))
        out = [np.empty(good.n, t) for t in (np.int32, np.int32, np.int64, np.int32)]
        nc = ctx.cluster(good.points, 900, 2, 2000, *out)
    np.testing.assert_array_equal(out[0], ref[0])
    np.testing.assert_array_equal(out[1], ref[1])
    np.testing.assert_array_equal(out[3], ref[3][0][0])
    assert nc == ref[3][0][1]
