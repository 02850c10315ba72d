"""Pins for the CPU oracle (no GPU needed).

The oracle is checked against things other than itself: hand-worked examples
(tests/golden/hand_worked.json, each derived from the paper's Definitions 1-6),
closed forms on integer lattices, invariants the definitions imply, and an
independent numpy brute force on small inputs. A last group plants mistakes in
copies of the oracle's C source and checks that these pins catch them.
"""
import ctypes
import json
import os
import subprocess

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_worked.json")
I64MAX = np.iinfo(np.int64).max


def _golden_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_golden_hand_worked(case):
    pts = np.array(case["points"], dtype=np.int32)
    rho = oracle.rho(pts, case["d_cut"])
    assert rho.tolist() == case["rho"]
    dep, d2 = oracle.dependent(pts, rho)
    assert dep.tolist() == case["dep"]
    assert d2.tolist() == case["delta2"]
    for q in case["queries"]:
        lab, nc = oracle.label(rho, dep, d2, q["rho_min"], q["delta_min"])
        assert lab.tolist() == q["label"], q["why"]
        assert nc == q["n_centers"], q["why"]


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("N,c", [(1, 1), (7, 1), (50, 3), (200, 17), (64, 64), (10, 100)])
def test_rho_line_lattice_closed_form(N, c):
    """x = 0..N-1 on a line: rho_i = min(i, c-1) + min(N-1-i, c-1) + 1."""
    pts = np.arange(N, dtype=np.int32).reshape(-1, 1)
    i = np.arange(N)
    expect = np.minimum(i, c - 1) + np.minimum(N - 1 - i, c - 1) + 1
    assert np.array_equal(oracle.rho(pts, c), expect)


@pytest.mark.parametrize("c", [1, 2, 3, 5, 7])
def test_rho_plane_lattice_gauss_circle(c):
    """Interior points of an integer grid see the Gauss circle count
    #{(a, b) in Z^2 : a^2 + b^2 < c^2}, enumerated over offsets."""
    L = 2 * c + 7
    xs, ys = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    pts = np.stack([xs.ravel(), ys.ravel()], axis=1).astype(np.int32)
    gauss = sum(1 for a in range(-c, c + 1) for b in range(-c, c + 1) if a * a + b * b < c * c)
    rho = oracle.rho(pts, c).reshape(L, L)
    inner = rho[c:L - c, c:L - c]
    assert inner.size > 0 and np.all(inner == gauss)


def test_rho_all_identical_points():
    pts = np.full((37, 3), 12345, dtype=np.int32)
    assert np.all(oracle.rho(pts, 1) == 37)
    dep, d2 = oracle.dependent(pts, oracle.rho(pts, 1))
    # identical densities: everyone depends on index 0 at distance 0
    assert dep[0] == -1 and d2[0] == I64MAX
    assert np.all(dep[1:] == 0) and np.all(d2[1:] == 0)


# ------------------------------------------------------------------ invariants

def _random_blobs(seed, n, d, spread=3000, dom=20000):
    rng = np.random.default_rng(seed)
    k = rng.integers(1, 5)
    cen = rng.integers(0, dom, size=(k, d))
    lab = rng.integers(0, k, size=n)
    pts = cen[lab] + rng.normal(0, spread, size=(n, d))
    pts = np.clip(np.rint(pts), 0, dom).astype(np.int32)
    # a few exact duplicates to exercise zero distances and ties
    if n > 10:
        pts[-3:] = pts[:3]
    return pts


@pytest.mark.parametrize("seed,n,d,dc", [(1, 300, 2, 900), (2, 500, 3, 1500), (3, 200, 8, 4000),
                                         (4, 400, 1, 50), (5, 257, 4, 2500)])
def test_rho_invariants(seed, n, d, dc):
    pts = _random_blobs(seed, n, d)
    rho = oracle.rho(pts, dc)
    assert rho.min() >= 1
    assert (int(rho.sum()) - n) % 2 == 0  # every unordered pair inside counts twice
    # translation invariance and permutation equivariance
    assert np.array_equal(oracle.rho(pts + 77, dc), rho)
    perm = np.random.default_rng(seed).permutation(n)
    assert np.array_equal(oracle.rho(pts[perm], dc), rho[perm])
    # subset form agrees
    idx = np.random.default_rng(seed + 1).choice(n, size=min(n, 50), replace=False)
    assert np.array_equal(oracle.rho_subset(pts, dc, idx), rho[idx])


def test_rank_order_is_lexicographic():
    rho = np.random.default_rng(7).integers(1, 6, size=1000).astype(np.int32)
    order = oracle.rank_order(rho)
    # numpy's lexsort on (index asc, rho desc) is the library special case
    expect = np.lexsort((np.arange(1000), -rho.astype(np.int64)))
    assert np.array_equal(order, expect)


def _brute_dependent(pts, rho):
    """Independent formulation: per point, mask the higher points and take the
    lexicographic minimum of (D, j); no sorting of the point set."""
    n = pts.shape[0]
    P = pts.astype(np.int64)
    dep = np.full(n, -1, dtype=np.int32)
    d2 = np.full(n, I64MAX, dtype=np.int64)
    idx = np.arange(n)
    for i in range(n):
        hi = (rho > rho[i]) | ((rho == rho[i]) & (idx < i))
        if not hi.any():
            continue
        D = ((P[hi] - P[i]) ** 2).sum(axis=1)
        js = idx[hi]
        m = D.min()
        j = js[D == m].min()
        dep[i], d2[i] = j, m
    return dep, d2


@pytest.mark.parametrize("seed,n,d,dc", [(11, 400, 2, 700), (12, 600, 3, 1200), (13, 300, 8, 5000),
                                         (14, 1500, 2, 300), (15, 350, 5, 3000)])
def test_dependent_against_brute_force(seed, n, d, dc):
    pts = _random_blobs(seed, n, d)
    rho = oracle.rho(pts, dc)
    dep, d2 = oracle.dependent(pts, rho)
    bdep, bd2 = _brute_dependent(pts, rho)
    assert np.array_equal(dep, bdep)
    assert np.array_equal(d2, bd2)
    # exactly one top point, and dependents rank strictly higher
    order = oracle.rank_order(rho)
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n)
    assert (dep == -1).sum() == 1 and dep[order[0]] == -1
    nz = dep >= 0
    assert np.all(rank[dep[nz]] < rank[nz])
    # a higher point inside the ball forces delta < d_cut
    P = pts.astype(np.int64)
    for i in np.random.default_rng(seed).choice(n, 40, replace=False):
        hi = (rho > rho[i]) | ((rho == rho[i]) & (np.arange(n) < i))
        if hi.any() and (((P[hi] - P[i]) ** 2).sum(axis=1) < dc * dc).any():
            assert d2[i] < dc * dc
    # subset form agrees with the prefix scan
    idx = np.random.default_rng(seed + 2).choice(n, 60, replace=False)
    sdep, sd2 = oracle.dependent_subset(pts, rho, idx)
    assert np.array_equal(sdep, dep[idx]) and np.array_equal(sd2, d2[idx])


def _chain_labels(rho, dep, d2, rho_min, delta_min):
    """Independent label formulation: follow dependent links to a center."""
    n = rho.shape[0]
    center = (rho >= rho_min) & (d2 >= delta_min * delta_min)
    lab = np.full(n, -1, dtype=np.int32)
    for i in range(n):
        if rho[i] < rho_min:
            continue
        p = i
        while not center[p]:
            p = dep[p]
        lab[i] = p
    return lab, int(center.sum())


@pytest.mark.parametrize("seed,n,d,dc,rmin,dmin", [(21, 500, 2, 900, 3, 3000), (22, 800, 3, 1500, 5, 4000),
                                                  (23, 300, 8, 5000, 2, 9000), (24, 400, 2, 600, 1, 700)])
def test_labels_against_chain_walk(seed, n, d, dc, rmin, dmin):
    pts = _random_blobs(seed, n, d)
    r = oracle.run(pts, dc, rmin, dmin)
    lab, nc = _chain_labels(r["rho"], r["dep"], r["delta2"], rmin, dmin)
    assert np.array_equal(r["label"], lab)
    assert r["n_centers"] == nc
    # noise is exactly rho < rho_min; centers label themselves; non-centers
    # share their dependent point's label (the forest rooted at centers)
    noise = r["rho"] < rmin
    assert np.array_equal(r["label"] == -1, noise)
    ctr = ~noise & (r["delta2"] >= dmin * dmin)
    assert np.all(r["label"][ctr] == np.nonzero(ctr)[0])
    mid = ~noise & ~ctr
    assert np.all(r["label"][mid] == r["label"][r["dep"][mid]])


def test_two_far_blobs_two_centers():
    rng = np.random.default_rng(3)
    a = rng.normal(10000, 300, size=(300, 2))
    b = rng.normal(60000, 300, size=(300, 2))
    pts = np.clip(np.rint(np.concatenate([a, b])), 0, 100000).astype(np.int32)
    r = oracle.run(pts, 200, 1, 20000)
    assert r["n_centers"] == 2
    assert len(set(r["label"][:300].tolist())) == 1
    assert len(set(r["label"][300:].tolist())) == 1
    assert r["label"][0] != r["label"][300]


# ------------------------------------------------- planted mistakes get caught

MUTATIONS = {
    "non_strict_cutoff": ("if (sq_dist(P, d, i, j) < r2) ++c;", "if (sq_dist(P, d, i, j) <= r2) ++c;"),
    "self_excluded": ("if (sq_dist(P, d, i, j) < r2) ++c;", "if (j != i && sq_dist(P, d, i, j) < r2) ++c;"),
    "tie_to_largest": ("if (dij < best_d || (dij == best_d && j < best_j)) {",
                       "if (dij < best_d || (dij == best_d && j > best_j)) {"),
    "strict_center": ("const int center = !noise && delta2[c] >= dmin2;",
                      "const int center = !noise && delta2[c] > dmin2;"),
    "dropped_dim": ("for (int32_t k = 0; k < d; ++k) {", "for (int32_t k = 1; k < d; ++k) {"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "dpc_oracle.c")).read()
    assert src.count(old) >= 1
    mut = src.replace(old, new)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(mut)
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-std=c99", str(c), "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.oracle_rho.argtypes = [vp, i64, i32, i64, vp]
    lib.oracle_dependent.argtypes = [vp, i64, i32, vp, vp, vp]
    lib.oracle_label.argtypes = [i64, vp, vp, vp, i64, i64, vp]
    lib.oracle_label.restype = i64
    return lib


def _golden_passes(lib):
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    for case in _golden_cases():
        pts = np.ascontiguousarray(case["points"], dtype=np.int32)
        n, d = pts.shape
        rho = np.empty(n, np.int32)
        lib.oracle_rho(p(pts), n, d, case["d_cut"], p(rho))
        dep = np.empty(n, np.int32)
        d2 = np.empty(n, np.int64)
        lib.oracle_dependent(p(pts), n, d, p(rho), p(dep), p(d2))
        if rho.tolist() != case["rho"] or dep.tolist() != case["dep"] or d2.tolist() != case["delta2"]:
            return False
        for q in case["queries"]:
            lab = np.empty(n, np.int32)
            nc = lib.oracle_label(n, p(rho), p(dep), p(d2), q["rho_min"], q["delta_min"], p(lab))
            if lab.tolist() != q["label"] or nc != q["n_centers"]:
                return False
    return True


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    lib = _build_mutant(tmp_path, name, old, new)
    assert not _golden_passes(lib), f"mutation {name} slipped past the hand-worked pins"


def test_unmutated_copy_passes(tmp_path):
    lib = _build_mutant(tmp_path, "identity", "int oracle_threads", "int oracle_threads")
    assert _golden_passes(lib)
