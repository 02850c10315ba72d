"""Approx-DPC on the GPU (Section 4.3) against the Approx-DPC oracle: the
hand-worked cases, random shapes element by element, seeded samples of the
full-size sets, the cluster-center guarantee against the exact path, and
switching between exact and approximate dependent points on one dataset."""
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


def run_approx(dpc, pts, d_cut, queries):
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    n = pts.shape[0]
    with dpc.Context(0) as ctx:
        rho = np.full(n, -7, np.int32)
        ds = ctx.density(pts, d_cut, rho)
        dep = np.full(n, -7, np.int32)
        d2 = np.full(n, -7, np.int64)
        ex = np.full(n, 7, np.uint8)
        ds.dependent_approx(dep, d2, ex)
        labs = []
        for rmin, dmin in queries:
            lab = np.full(n, -7, np.int32)
            labs.append((lab, ds.label(rmin, dmin, lab)))
        info = ds.info()
        ds.release()
    return rho, dep, d2, ex, labs, info


def test_golden_cases(dpc):
    with open(os.path.join(os.path.dirname(__file__), "golden", "approx_hand_worked.json")) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        q = [(x["rho_min"], x["delta_min"]) for x in case["queries"]]
        rho, dep, d2, ex, labs, _ = run_approx(dpc, case["points"], case["d_cut"], q)
        assert rho.tolist() == case["rho"], case["name"]
        assert dep.tolist() == case["dep"], case["name"]
        assert d2.tolist() == case["delta2"], case["name"]
        assert ex.tolist() == case["exact"], case["name"]
        for (lab, nc), x in zip(labs, case["queries"]):
            assert lab.tolist() == x["label"] and nc == x["n_centers"], (case["name"], x["why"])


SHAPES = [
    (1, 2000, 2, 1000, 100000, 4, 0.05, 0),
    (2, 3000, 3, 2500, 100000, 5, 0.04, 20),
    (3, 2500, 1, 40, 100000, 6, 0.01, 25),
    (4, 1500, 4, 6000, 100000, 3, 0.05, 0),
    (5, 1200, 5, 9000, 100000, 3, 0.05, 0),
    (6, 1500, 8, 9000, 100000, 5, 0.05, 20),
    (7, 4000, 3, 1, 50, 2, 0.2, 100),       # d_cut = 1: side 1
    (8, 5000, 2, 30, 1000, 3, 0.2, 50),     # many points per cell
    (9, 2000, 3, 200, 100000, 40, 0.002, 0),
    (10, 3000, 4, 2, 30, 3, 0.2, 50),      # corner cells of the d_cut grid left out
    (11, 2500, 8, 3, 12, 3, 0.3, 30),
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"n{s[1]}_d{s[2]}_dc{s[3]}")
def test_random_shapes_bit_exact(dpc, shape):
    seed, n, d, dc, dom, blobs, spread, dup = shape
    ds = workloads.random_blobs(seed, n, d, dc, domain=dom, blobs=blobs, spread=spread, dup=dup)
    q = [(2, dc + 1), (1, 3 * dc + 1), (5, 10 * dc)]
    rho, dep, d2, ex, labs, _ = run_approx(dpc, ds.points, dc, q)
    orho = oracle.rho(ds.points, dc)
    np.testing.assert_array_equal(rho, orho)
    odep, od2, oex = oracle.approx_dependent(ds.points, orho, dc)
    np.testing.assert_array_equal(dep, odep)
    np.testing.assert_array_equal(d2, od2)
    np.testing.assert_array_equal(ex.astype(bool), oex)
    for (lab, nc), (rmin, dmin) in zip(labs, q):
        olab, onc = oracle.label(orho, odep, od2, rmin, dmin)
        np.testing.assert_array_equal(lab, olab)
        assert nc == onc


def test_high_dims_finer_grid(dpc):
    """Approx-DPC on an 8-d set with the exact grid's cells of side d_cut / 2."""
    ds = workloads.random_blobs(6, 1500, 8, 9000, blobs=5, spread=0.05, dup=20)
    pts = np.ascontiguousarray(ds.points)
    n = pts.shape[0]
    with dpc.Context(0) as ctx:
        ctx.tune(hd_cell_factor=2, hd_min_d=5)
        rho = np.empty(n, np.int32)
        h = ctx.density(pts, 9000, rho)
        dep = np.empty(n, np.int32)
        d2 = np.empty(n, np.int64)
        ex = np.empty(n, np.uint8)
        h.dependent_approx(dep, d2, ex)
        h.release()
    orho = oracle.rho(pts, 9000)
    odep, od2, oex = oracle.approx_dependent(pts, orho, 9000)
    np.testing.assert_array_equal(rho, orho)
    np.testing.assert_array_equal(dep, odep)
    np.testing.assert_array_equal(d2, od2)
    np.testing.assert_array_equal(ex.astype(bool), oex)


def test_identical_points_and_tiny(dpc):
    for pts, dc in [(np.full((500, 3), 77, np.int32), 5), (np.array([[3, 4]], np.int32), 2),
                    (np.array([[0, 0], [0, 1]], np.int32), 2)]:
        rho, dep, d2, ex, labs, _ = run_approx(dpc, pts, dc, [(1, dc + 1)])
        orho = oracle.rho(pts, dc)
        odep, od2, oex = oracle.approx_dependent(pts, orho, dc)
        np.testing.assert_array_equal(dep, odep)
        np.testing.assert_array_equal(d2, od2)
        np.testing.assert_array_equal(ex.astype(bool), oex)


def test_exact_and_approx_on_one_dataset(dpc):
    """dpc_label follows whichever dependent points were computed last."""
    ds = workloads.random_blobs(33, 3000, 2, 1500, blobs=4, spread=0.05)
    pts = ds.points
    n = pts.shape[0]
    r = oracle.run(pts, 1500, 2, 4000)
    a = oracle.run_approx(pts, 1500, 2, 4000)
    with dpc.Context(0) as ctx:
        h = ctx.density(pts, 1500)
        lab = np.empty(n, np.int32)
        h.dependent_approx()
        assert h.label(2, 4000, lab) == a["n_centers"]
        np.testing.assert_array_equal(lab, a["label"])
        dep = np.empty(n, np.int32)
        h.dependent(dep)
        np.testing.assert_array_equal(dep, r["dep"])
        assert h.label(2, 4000, lab) == r["n_centers"]
        np.testing.assert_array_equal(lab, r["label"])
        h.dependent_approx()
        h.label(2, 4000, lab)
        np.testing.assert_array_equal(lab, a["label"])
        h.release()


def check_sampled(dpc, ds, m, seed):
    pts = ds.points
    n = ds.n
    q = [(ds.rho_min, ds.delta_min)]
    rho, dep, d2, ex, labs, info = run_approx(dpc, pts, ds.d_cut, q)
    idx = np.sort(np.random.default_rng(seed).choice(n, size=min(m, n), replace=False))
    np.testing.assert_array_equal(rho[idx], oracle.rho_subset(pts, ds.d_cut, idx))
    sdep, sd2, sex = oracle.approx_dependent_subset(pts, rho, ds.d_cut, idx)
    np.testing.assert_array_equal(dep[idx], sdep)
    np.testing.assert_array_equal(d2[idx], sd2)
    np.testing.assert_array_equal(ex[idx].astype(bool), sex)
    # every point: links go to higher points; approximated ones carry d_cut
    order = oracle.rank_order(rho)
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    assert dep[order[0]] == -1 and d2[order[0]] == I64MAX
    nz = dep >= 0
    assert np.all(rank[dep[nz]] < rank[nz])
    assert np.all(d2[~ex.astype(bool)] == ds.d_cut * ds.d_cut)
    # labels from the GPU links (oracle step 4) and the center guarantee:
    # the centers are those of the exact path
    lab, nc = labs[0]
    olab, onc = oracle.label(rho, dep, d2, ds.rho_min, ds.delta_min)
    np.testing.assert_array_equal(lab, olab)
    assert nc == onc
    with dpc.Context(0) as ctx:
        h = ctx.density(pts, ds.d_cut)
        elab = np.empty(n, np.int32)
        enc = h.label(ds.rho_min, ds.delta_min, elab)
        h.release()
    assert nc == enc
    np.testing.assert_array_equal(np.nonzero(lab == np.arange(n))[0], np.nonzero(elab == np.arange(n))[0])
    return info


def test_plain_1m_8d_sampled(dpc):
    check_sampled(dpc, workloads.plain_1m_8d(), 1000, 41)


def test_plain_5p8m_3d_sampled(dpc):
    check_sampled(dpc, workloads.plain_5p8m_3d(), 2000, 42)
