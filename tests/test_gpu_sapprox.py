"""S-Approx-DPC on the GPU (Section 5) against the S-Approx-DPC oracle: the
hand-worked cases, random shapes element by element for several eps, keys of
G' wider than 64 bits, the reduction to exact DPC on cells of one point,
edge cases, host and device buffers, and seeded samples of the full-size
sets."""
import json
import os

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


def run_sapprox(dpc, pts, d_cut, eps, queries, knobs=None):
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    n = pts.shape[0]
    with dpc.Context(0) as ctx:
        if knobs:
            ctx.tune(**knobs)
        rho = np.full(n, -7, np.int32)
        dep = np.full(n, -7, np.int32)
        d2 = np.full(n, -7, np.int64)
        pk = np.full(n, 7, np.uint8)
        ds = ctx.sapprox(pts, d_cut, eps, rho, dep, d2, pk)
        labs = []
        for rmin, dmin in queries:
            lab = np.full(n, -7, np.int32)
            labs.append((lab, ds.label(rmin, dmin, lab)))
        info = ds.info()
        ds.release()
    return rho, dep, d2, pk.astype(bool), labs, info


def check_full(dpc, pts, dc, eps, queries, knobs=None):
    num, den = eps
    rho, dep, d2, pk, labs, info = run_sapprox(dpc, pts, dc, eps, queries, knobs)
    orho, odep, od2, opk = oracle.sapprox(pts, dc, num, den)
    np.testing.assert_array_equal(pk, opk)
    np.testing.assert_array_equal(rho, orho)
    np.testing.assert_array_equal(dep, odep)
    np.testing.assert_array_equal(d2, od2)
    for (lab, nc), (rmin, dmin) in zip(labs, queries):
        olab, onc = oracle.sapprox_label(orho, odep, od2, opk, rmin, dmin)
        np.testing.assert_array_equal(lab, olab)
        assert nc == onc
    assert info["picks"] == int(opk.sum())
    return info


def test_golden_cases(dpc):
    with open(os.path.join(os.path.dirname(__file__), "golden", "sapprox_hand_worked.json")) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        q = [(x["rho_min"], x["delta_min"]) for x in case["queries"]]
        rho, dep, d2, pk, labs, _ = run_sapprox(dpc, case["points"], case["d_cut"],
                                                (case["eps_num"], case["eps_den"]), q)
        assert rho.tolist() == case["rho"], case["name"]
        assert dep.tolist() == case["dep"], case["name"]
        assert d2.tolist() == case["delta2"], case["name"]
        assert pk.astype(int).tolist() == case["pick"], case["name"]
        for (lab, nc), x in zip(labs, case["queries"]):
            assert lab.tolist() == x["label"] and nc == x["n_centers"], (case["name"], x["why"])


SHAPES = [
    # seed, n, d, d_cut, domain, blobs, spread, dup
    (1, 2000, 2, 1000, 100000, 4, 0.05, 0),
    (2, 3000, 3, 2500, 100000, 5, 0.04, 20),
    (3, 2500, 1, 40, 100000, 6, 0.01, 25),
    (4, 1500, 4, 6000, 100000, 3, 0.05, 0),
    (5, 1200, 5, 9000, 100000, 3, 0.05, 0),
    (6, 1500, 8, 9000, 100000, 5, 0.05, 20),
    (7, 4000, 3, 1, 50, 2, 0.2, 100),       # d_cut = 1: side 1
    (8, 5000, 2, 30, 1000, 3, 0.2, 50),     # many points per cell
    (9, 2000, 3, 200, 100000, 40, 0.002, 0),
    (10, 3000, 4, 2, 30, 3, 0.2, 50),      # cells left out of the neighbour runs
    (11, 2500, 8, 3, 12, 3, 0.3, 30),
]
EPS = [(4, 5), (1, 5), (1, 1), (3, 1)]


@pytest.mark.parametrize("eps", EPS, ids=lambda e: f"eps{e[0]}_{e[1]}")
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"n{s[1]}_d{s[2]}_dc{s[3]}")
def test_random_shapes_bit_exact(dpc, shape, eps):
    seed, n, d, dc, dom, blobs, spread, dup = shape
    ds = workloads.random_blobs(seed, n, d, dc, domain=dom, blobs=blobs, spread=spread, dup=dup)
    check_full(dpc, ds.points, dc, eps, [(2, dc + 1), (1, 3 * dc + 1), (5, 10 * dc)])


def test_high_dims_finer_exact_grid(dpc):
    """The density and first-phase scans over an exact grid of side d_cut / 2."""
    ds = workloads.random_blobs(6, 1500, 8, 9000, blobs=5, spread=0.05, dup=20)
    check_full(dpc, ds.points, 9000, (4, 5), [(2, 9001)], knobs={"hd_cell_factor": 2, "hd_min_d": 5})


def test_keys_wider_than_64_bits(dpc):
    """8 dims over a wide domain with a small side: the key of G' needs more
    than one 64-bit word (three sort passes here)."""
    rng = np.random.default_rng(71)
    pts = rng.integers(0, 1 << 29, size=(3000, 8)).astype(np.int32)
    pts[1000:1500] = pts[:500] + rng.integers(-3, 4, size=(500, 8)).astype(np.int32)
    pts = np.clip(pts, 0, (1 << 30) - 1)
    dc = 40
    s = oracle.sapprox_side(dc, 8, 1, 1)
    span = pts.max(0).astype(np.int64) - pts.min(0) + 1
    assert sum(int((x - 1) // s).bit_length() for x in span) > 128
    check_full(dpc, pts, dc, (1, 1), [(1, dc + 1), (2, 50 * dc)])


def test_unit_cells_match_exact(dpc):
    """Side 1 on distinct points: S-Approx-DPC is exact DPC."""
    rng = np.random.default_rng(5)
    pts = np.unique(rng.integers(0, 3000, size=(20000, 2)), axis=0).astype(np.int32)
    rng.shuffle(pts)
    dc = 60
    rho, dep, d2, pk, _, _ = run_sapprox(dpc, pts, dc, (1, 10 ** 6), [])
    assert pk.all()
    r = oracle.run(pts, dc, 2, dc + 1)
    np.testing.assert_array_equal(rho, r["rho"])
    np.testing.assert_array_equal(dep, r["dep"])
    np.testing.assert_array_equal(d2, r["delta2"])


def test_edge_cases(dpc):
    cases = [
        (np.full((500, 3), 77, np.int32), 5),             # one cell, one pick
        (np.array([[3, 4]], np.int32), 2),                 # a single point
        (np.array([[0, 0], [0, 1]], np.int32), 2),
        (np.array([[0], [1 << 29], [(1 << 30) - 1]], np.int32), 1),  # far apart, side 1
    ]
    for pts, dc in cases:
        for eps in [(1, 1), (1, 5), (7, 1)]:
            check_full(dpc, pts, dc, eps, [(1, dc + 1)])
    with dpc.Context(0) as ctx:
        h = ctx.sapprox(np.zeros((0, 3), np.int32), 5, (1, 1))
        assert h.label(1, 6) == 0
        h.release()


def test_device_buffers_and_dataset_calls(dpc):
    import torch
    ds = workloads.random_blobs(44, 4000, 3, 2500, blobs=5, spread=0.04, dup=10)
    pts = ds.points
    n = pts.shape[0]
    orho, odep, od2, opk = oracle.sapprox(pts, 2500, 4, 5)
    olab, onc = oracle.sapprox_label(orho, odep, od2, opk, 3, 6000)
    dev = torch.device("cuda", 0)
    tp = torch.from_numpy(pts).to(dev)
    rho = torch.empty(n, dtype=torch.int32, device=dev)
    dep = torch.empty(n, dtype=torch.int32, device=dev)
    d2 = torch.empty(n, dtype=torch.int64, device=dev)
    pk = torch.empty(n, dtype=torch.uint8, device=dev)
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    with dpc.Context(0) as ctx:
        h = ctx.sapprox(tp, 2500, 0.8, rho, dep, d2, pk)
        nc = h.label(3, 6000, lab)
        # dpc_dependent copies the same dependent points; Approx-DPC's are refused
        dep2 = torch.empty(n, dtype=torch.int32, device=dev)
        h.dependent(dep2)
        with pytest.raises(dpc.DpcError):
            h.dependent_approx()
        ctx.stream.synchronize()
        h.release()
    np.testing.assert_array_equal(rho.cpu().numpy(), orho)
    np.testing.assert_array_equal(dep.cpu().numpy(), odep)
    np.testing.assert_array_equal(dep2.cpu().numpy(), odep)
    np.testing.assert_array_equal(d2.cpu().numpy(), od2)
    np.testing.assert_array_equal(pk.cpu().numpy().astype(bool), opk)
    np.testing.assert_array_equal(lab.cpu().numpy(), olab)
    assert nc == onc


def test_cluster_sapprox_helper(dpc):
    ds = workloads.random_blobs(45, 3000, 2, 1500, blobs=4, spread=0.05)
    r = dpc.cluster_sapprox(ds.points, 1500, (3, 5), 2, 4000)
    orho, odep, od2, opk = oracle.sapprox(ds.points, 1500, 3, 5)
    olab, onc = oracle.sapprox_label(orho, odep, od2, opk, 2, 4000)
    np.testing.assert_array_equal(r["label"], olab)
    assert r["n_centers"] == onc


def check_sampled(dpc, ds, eps, m, seed):
    pts = ds.points
    n = ds.n
    num, den = eps
    q = [(ds.rho_min, ds.delta_min)]
    rho, dep, d2, pk, labs, info = run_sapprox(dpc, pts, ds.d_cut, eps, q)
    idx = np.sort(np.random.default_rng(seed).choice(n, size=min(m, n), replace=False))
    # the sampled points' picks, links and (for picks) densities
    sdep, sd2, spk = oracle.sapprox_dependent_subset(pts, np.where(pk, rho, 0), ds.d_cut, num, den, idx)
    np.testing.assert_array_equal(pk[idx], spk)
    np.testing.assert_array_equal(dep[idx], sdep)
    np.testing.assert_array_equal(d2[idx], sd2)
    sp = idx[pk[idx]]
    np.testing.assert_array_equal(rho[sp], oracle.rho_subset(pts, ds.d_cut, sp))
    assert np.all(rho[~pk] == -1)
    # every point: picks link to higher picks, the others to a pick
    assert info["picks"] == int(pk.sum())
    picks = np.nonzero(pk)[0]
    key = np.lexsort((picks, -rho[picks].astype(np.int64)))
    rank = np.full(n, n, np.int64)
    rank[picks[key]] = np.arange(picks.size)
    top = picks[key[0]]
    assert dep[top] == -1 and d2[top] == I64MAX
    others = np.nonzero(pk & (np.arange(n) != top))[0]
    assert np.all(pk[dep[others]]) and np.all(rank[dep[others]] < rank[others])
    nop = np.nonzero(~pk)[0]
    assert np.all(pk[dep[nop]])
    # labels from the GPU links (the oracle's label step)
    lab, nc = labs[0]
    olab, onc = oracle.sapprox_label(rho, dep, d2, pk, ds.rho_min, ds.delta_min)
    np.testing.assert_array_equal(lab, olab)
    assert nc == onc
    return info


def test_plain_5p8m_3d_sampled(dpc):
    check_sampled(dpc, workloads.plain_5p8m_3d(), (4, 5), 1500, 51)


def test_plain_1m_8d_sampled(dpc):
    check_sampled(dpc, workloads.plain_1m_8d(), (1, 5), 600, 52)


def test_both_paths_by_pair_counts(dpc):
    """Few picks facing many candidates: the pick path (no all-point density
    pairs); many picks: the all-point path."""
    few = workloads.random_blobs(8, 5000, 2, 30, domain=1000, blobs=3, spread=0.2, dup=50)
    info = check_full(dpc, few.points, 30, (3, 1), [(2, 31)])
    assert info["dense_pairs"] == 0
    many = workloads.random_blobs(1, 2000, 2, 1000, domain=100000, blobs=4, spread=0.05)
    info = check_full(dpc, many.points, 1000, (1, 5), [(2, 1001)])
    assert info["dense_pairs"] > 0


@pytest.mark.parametrize("path,by_cell,near_threads", [(1, 1, 1), (2, 1, 1), (2, 0, 1), (2, 1, 0), (2, 3, 1)])
@pytest.mark.parametrize("shape", [SHAPES[i] for i in (1, 3, 5, 6, 7, 9, 10)], ids=lambda s: f"n{s[1]}_d{s[2]}_dc{s[3]}")
def test_forced_paths(dpc, shape, path, by_cell, near_threads):
    """Either path (the pick path's density by cell, by pick or in the dense
    kernels over pick items, its near pass by thread or by warp) on any data
    gives the oracle's bits."""
    seed, n, d, dc, dom, blobs, spread, dup = shape
    ds = workloads.random_blobs(seed, n, d, dc, domain=dom, blobs=blobs, spread=spread, dup=dup)
    for eps in [(4, 5), (3, 1)]:
        check_full(dpc, ds.points, dc, eps, [(2, dc + 1), (1, 3 * dc + 1)],
                   knobs={"sapprox_path": path, "sapprox_rho_cells": by_cell, "sapprox_near_threads": near_threads})


@pytest.mark.parametrize("eps", [(1, 20), (1, 5)], ids=lambda e: f"eps{e[0]}_{e[1]}")
@pytest.mark.parametrize("kch", [64, 2048])
def test_pick_items_chunks(dpc, eps, kch):
    """The pick path's density in the dense kernels over pick items: cells
    with more than 128 picks (several pick chunks per cell, small eps) and
    items of 64 candidates (several candidate chunks) give the oracle's
    bits, and the info names the path."""
    ds = workloads.random_blobs(91, 6000, 3, 400, domain=20000, blobs=3, spread=0.01, dup=4)
    info = check_full(dpc, ds.points, 400, eps, [(2, 401), (1, 1201)],
                      knobs={"sapprox_path": 2, "sapprox_rho_cells": 3, "kch": kch})
    assert info["density_path"] == 3
    assert info["dense_pairs"] == info["cand_pairs"] > 0


def test_density_path_reported(dpc):
    """dpc_info.density_path follows the path each call took."""
    ds = workloads.random_blobs(92, 3000, 2, 300, domain=30000, blobs=3, spread=0.03, dup=2)
    for knobs, path in [({"sapprox_path": 1}, 0), ({"sapprox_path": 2, "sapprox_rho_cells": 0}, 1),
                        ({"sapprox_path": 2, "sapprox_rho_cells": 1}, 2),
                        ({"sapprox_path": 2, "sapprox_rho_cells": 3}, 3)]:
        info = check_full(dpc, ds.points, 300, (4, 5), [(2, 301)], knobs=knobs)
        assert info["density_path"] == path, knobs
