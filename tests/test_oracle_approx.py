"""Pins of the Approx-DPC oracle (Section 4.3), independent of the oracle's
own code: hand-worked cases, the paper's cluster-center guarantee (Section
4.4: the same centers as the exact algorithm whenever delta_min > d_cut),
geometric and rank properties of every approximate link, equality with the
exact oracle wherever the dependent point is computed exactly, the sampled
form against the full one, and planted mistakes that the hand-worked cases
must catch."""
import ctypes
import json
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "approx_hand_worked.json")


def _cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_hand_worked(case):
    pts = np.array(case["points"], dtype=np.int32)
    assert oracle.approx_side(case["d_cut"], pts.shape[1]) == case["side"]
    rho = oracle.rho(pts, case["d_cut"])
    assert rho.tolist() == case["rho"]
    dep, d2, ex = oracle.approx_dependent(pts, rho, case["d_cut"])
    assert dep.tolist() == case["dep"]
    assert d2.tolist() == case["delta2"]
    assert ex.astype(int).tolist() == case["exact"]
    for q in case["queries"]:
        lab, nc = oracle.label(rho, dep, d2, q["rho_min"], q["delta_min"])
        assert lab.tolist() == q["label"] and nc == q["n_centers"], q["why"]


def test_side_closed_form():
    # floor(d_cut / sqrt(d)), at least 1, for the sizes the workloads use
    for d_cut in (1, 2, 3, 5, 100, 178, 1000, 4040):
        for d in range(1, 9):
            s = oracle.approx_side(d_cut, d)
            assert s == max(1, math.isqrt(d_cut * d_cut // d))
            # the defining property: s * sqrt(d) <= d_cut < (s + 1) * sqrt(d), unless clamped at 1
            assert s * s * d <= d_cut * d_cut or s == 1
            assert (s + 1) * (s + 1) * d > d_cut * d_cut


SHAPES = [(11, 800, 1, 40), (12, 1500, 2, 900), (13, 2000, 2, 3000), (14, 1200, 3, 4000), (15, 900, 4, 9000),
          (16, 1000, 3, 300), (17, 600, 5, 12000)]


def _ranks(rho):
    order = np.lexsort((np.arange(rho.size), -rho.astype(np.int64)))
    rank = np.empty(rho.size, np.int64)
    rank[order] = np.arange(rho.size)
    return rank


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"n{s[1]}_d{s[2]}_dc{s[3]}")
def test_properties_against_the_exact_oracle(shape):
    seed, n, d, dc = shape
    ds = workloads.random_blobs(seed, n, d, dc, blobs=4, spread=0.05, dup=5)
    pts = ds.points
    rho = oracle.rho(pts, dc)
    dep, d2, ex = oracle.approx_dependent(pts, rho, dc)
    edep, ed2 = oracle.dependent(pts, rho)
    rank = _ranks(rho)
    P = pts.astype(np.int64)
    top = int(np.argmin(rank))
    assert dep[top] == -1 and d2[top] == np.iinfo(np.int64).max and ex[top]
    others = np.arange(n) != top
    # every link goes to a higher point
    assert np.all(rank[dep[others]] < rank[others])
    # exactly computed links are the exact oracle's
    np.testing.assert_array_equal(dep[ex], edep[ex])
    np.testing.assert_array_equal(d2[ex], ed2[ex])
    # approximated links carry delta = d_cut and, for points that are not
    # their cell's top, land within d_cut (same cell, side d_cut / sqrt(d))
    ap = ~ex
    assert np.all(d2[ap] == dc * dc)
    dd = ((P[ap] - P[dep[ap]]) ** 2).sum(axis=1)
    # a cell's own top is within d_cut; a top linked to another cell's top
    # may be farther, but some point of that cell is within d_cut
    s = oracle.approx_side(dc, d)
    cell = (P - P.min(axis=0)) // s
    same = np.all(cell[ap] == cell[dep[ap]], axis=1)
    assert np.all(dd[same] < dc * dc)
    for i in np.nonzero(ap)[0][~same]:
        in_c = np.all(cell == cell[dep[i]], axis=1)
        assert np.all(rank[in_c] < rank[i])        # every point of that cell is higher
        near = ((P[in_c] - P[i]) ** 2).sum(axis=1) < dc * dc
        assert near.any()                          # and one of them is within d_cut
    # an approximated point never has an exact delta above d_cut (that is
    # what makes the centers exact), and exact ones with delta <= d_cut only
    # occur when no higher point within d_cut exists in a qualifying cell
    assert np.all(ed2[ap] <= dc * dc)
    # the cluster-center guarantee (Section 4.4) for delta_min > d_cut
    for rmin, dmin in [(2, dc + 1), (3, 2 * dc), (1, 5 * dc)]:
        lab, nc = oracle.label(rho, dep, d2, rmin, dmin)
        elab, enc = oracle.label(rho, edep, ed2, rmin, dmin)
        assert nc == enc
        centers = set(np.nonzero(lab == np.arange(n))[0].tolist())
        ecenters = set(np.nonzero(elab == np.arange(n))[0].tolist())
        assert centers == ecenters
        np.testing.assert_array_equal(lab == -1, elab == -1)


def test_subset_matches_full():
    ds = workloads.random_blobs(21, 1500, 3, 2500, blobs=5, spread=0.04, dup=7)
    rho = oracle.rho(ds.points, 2500)
    dep, d2, ex = oracle.approx_dependent(ds.points, rho, 2500)
    idx = np.sort(np.random.default_rng(3).choice(1500, size=300, replace=False))
    sdep, sd2, sex = oracle.approx_dependent_subset(ds.points, rho, 2500, idx)
    np.testing.assert_array_equal(sdep, dep[idx])
    np.testing.assert_array_equal(sd2, d2[idx])
    np.testing.assert_array_equal(sex, ex[idx])


# ------------------------------------------------- planted mistakes get caught

MUTATIONS = {
    "side_without_sqrt_d": ("int64_t s = isqrt_i64((d_cut * d_cut) / d);", "int64_t s = d_cut;"),
    "non_strict_neighbourhood": ("if (cj == c || sq_dist(P, d, i, j) >= r2) continue;",
                                 "if (cj == c || sq_dist(P, d, i, j) > r2) continue;"),
    "lowest_point_as_top": ("if (rank[i] < rank[pstar[c]]) pstar[c] = i;", "if (rank[i] > rank[pstar[c]]) pstar[c] = i;"),
    "first_qualifying_cell": ("if (maxrank[cj] < rank[i] && (best < 0 || rank[pstar[cj]] < rank[best])) best = pstar[cj];",
                              "if (maxrank[cj] < rank[i] && best < 0) best = pstar[cj];"),
    "only_top_must_be_higher": ("if (maxrank[cj] < rank[i] && (best < 0 || rank[pstar[cj]] < rank[best])) best = pstar[cj];",
                                "if (rank[pstar[cj]] < rank[i] && (best < 0 || rank[pstar[cj]] < rank[best])) best = pstar[cj];"),
}


def _build(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "dpc_oracle.c")).read()
    assert src.count(old) == 1, name
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src.replace(old, new))
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-std=c99", str(c), "-o", str(so), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.oracle_rho.argtypes = [vp, i64, i32, i64, vp]
    lib.oracle_approx_dependent.argtypes = [vp, i64, i32, i64, vp, vp, vp, vp]
    return lib


def _golden_passes(lib):
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    for case in _cases():
        pts = np.ascontiguousarray(case["points"], dtype=np.int32)
        n, d = pts.shape
        rho = np.empty(n, np.int32)
        lib.oracle_rho(p(pts), n, d, case["d_cut"], p(rho))
        dep = np.empty(n, np.int32)
        d2 = np.empty(n, np.int64)
        ex = np.empty(n, np.int32)
        lib.oracle_approx_dependent(p(pts), n, d, case["d_cut"], p(rho), p(dep), p(d2), p(ex))
        if dep.tolist() != case["dep"] or d2.tolist() != case["delta2"] or ex.tolist() != case["exact"]:
            return False
    return True


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    assert not _golden_passes(_build(tmp_path, name, *MUTATIONS[name])), name


def test_unmutated_copy_passes(tmp_path):
    assert _golden_passes(_build(tmp_path, "identity", "int oracle_threads", "int oracle_threads"))
