"""Pins of the S-Approx-DPC oracle (Section 5), independent of its code:
hand-worked cases, the closed form of the grid side, the case where every
cell holds one distinct point (then S-Approx-DPC is exact DPC, so its links
must equal the exact oracle's), picks' densities equal to Definition 1,
every link going to a higher pick, second-phase links equal to a brute
force over the picks, and planted mistakes the hand-worked cases catch."""
import ctypes
import json
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sapprox_hand_worked.json")


def _cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_hand_worked(case):
    pts = np.array(case["points"], dtype=np.int32)
    assert oracle.sapprox_side(case["d_cut"], pts.shape[1], case["eps_num"], case["eps_den"]) == case["side"]
    rho, dep, d2, pk = oracle.sapprox(pts, case["d_cut"], case["eps_num"], case["eps_den"])
    assert rho.tolist() == case["rho"]
    assert dep.tolist() == case["dep"]
    assert d2.tolist() == case["delta2"]
    assert pk.astype(int).tolist() == case["pick"]
    for q in case["queries"]:
        lab, nc = oracle.sapprox_label(rho, dep, d2, pk, q["rho_min"], q["delta_min"])
        assert lab.tolist() == q["label"] and nc == q["n_centers"], q["why"]


def test_side_closed_form():
    for d_cut in (1, 5, 178, 1000, 4040):
        for d in range(1, 9):
            for num, den in [(1, 1), (1, 2), (3, 1), (7, 10), (1, 1000)]:
                s = oracle.sapprox_side(d_cut, d, num, den)
                exact = math.isqrt((num * num * d_cut * d_cut) // (den * den * d))
                assert s == max(1, exact)


@pytest.mark.parametrize("seed,d", [(1, 2), (2, 3), (3, 1)])
def test_unit_cells_equal_exact(seed, d):
    """Side 1 with distinct points: every point is a pick and S-Approx-DPC
    computes exact DPC (first phase: nearest higher point within d_cut;
    second phase: nearest higher point overall)."""
    rng = np.random.default_rng(seed)
    pts = np.unique(rng.integers(0, 400, size=(900, d)), axis=0).astype(np.int32)
    rng.shuffle(pts)
    dc = 30
    rho, dep, d2, pk = oracle.sapprox(pts, dc, 1, 10 ** 6)
    assert pk.all()
    erho = oracle.rho(pts, dc)
    edep, ed2 = oracle.dependent(pts, erho)
    np.testing.assert_array_equal(rho, erho)
    np.testing.assert_array_equal(dep, edep)
    np.testing.assert_array_equal(d2, ed2)


@pytest.mark.parametrize("seed,n,d,dc,num,den", [(11, 1500, 2, 900, 1, 1), (12, 2000, 3, 2500, 1, 2),
                                                 (13, 1200, 4, 6000, 2, 1), (14, 800, 6, 12000, 1, 1)])
def test_properties(seed, n, d, dc, num, den):
    ds = workloads.random_blobs(seed, n, d, dc, blobs=4, spread=0.05, dup=5)
    pts = ds.points
    P = pts.astype(np.int64)
    rho, dep, d2, pk = oracle.sapprox(pts, dc, num, den)
    s = oracle.sapprox_side(dc, d, num, den)
    cell = (P - P.min(axis=0)) // s
    # one pick per cell: its smallest index
    keys = [tuple(c) for c in cell.tolist()]
    first = {}
    for i, k in enumerate(keys):
        first.setdefault(k, i)
    np.testing.assert_array_equal(pk, np.array([first[k] == i for i, k in enumerate(keys)]))
    picks = np.nonzero(pk)[0]
    # densities of the picks: Definition 1 (the exact oracle's sampled form)
    np.testing.assert_array_equal(rho[picks], oracle.rho_subset(pts, dc, picks))
    assert np.all(rho[~pk] == -1)
    # points that are not picked depend on their cell's pick at their distance
    nop = np.nonzero(~pk)[0]
    np.testing.assert_array_equal(dep[nop], [first[keys[i]] for i in nop])
    np.testing.assert_array_equal(d2[nop], ((P[nop] - P[dep[nop]]) ** 2).sum(axis=1))
    # picks: links to higher picks, exact distances
    higher = lambda q, i: rho[q] > rho[i] or (rho[q] == rho[i] and q < i)
    top = [i for i in picks if dep[i] == -1]
    assert len(top) == 1
    for i in picks:
        if dep[i] < 0:
            continue
        assert pk[dep[i]] and higher(dep[i], i)
        assert d2[i] == ((P[i] - P[dep[i]]) ** 2).sum()
    # brute force of both phases with numpy: the candidates of the first
    # phase are the higher picks of the cells (other than its own) holding a
    # point strictly within d_cut of the pick; without candidates, the
    # nearest higher pick over all picks
    cell_id = np.array([first[k] for k in keys])
    for i in picks[:300]:
        if dep[i] < 0:
            continue
        near = ((P - P[i]) ** 2).sum(axis=1) < dc * dc
        cand = np.unique(cell_id[near & (cell_id != cell_id[i])])
        cand = np.array([q for q in cand if higher(q, i)], dtype=np.int64)
        if cand.size == 0:
            cand = np.array([q for q in picks if higher(q, i)], dtype=np.int64)
        dd = ((P[cand] - P[i]) ** 2).sum(axis=1)
        best = cand[dd == dd.min()].min()
        assert dep[i] == best and d2[i] == dd.min()


MUTATIONS = {
    "largest_index_pick": ("if (i < cpick[c]) cpick[c] = i;", "if (i > cpick[c]) cpick[c] = i;"),
    "farthest_first_phase": ("        if (dq < d2 || (dq == d2 && q < dp)) {\n            d2 = dq;\n            dp = q;\n        }\n    }\n    if (dp < 0) {",
                             "        if (dp < 0 || dq > d2) {\n            d2 = dq;\n            dp = q;\n        }\n    }\n    if (dp < 0) {"),
    "side_without_sqrt_d": ("const int64_t s = oracle_sapprox_side(d_cut, d, eps_num, eps_den);",
                            "const int64_t s = oracle_sapprox_side(d_cut, 1, eps_num, eps_den);"),
    "non_strict_neighbourhood": ("if (cell[j] == cell[i] || sq_dist(P, d, i, j) >= r2) continue;",
                                 "if (cell[j] == cell[i] || sq_dist(P, d, i, j) > r2) continue;"),
    "lower_picks_allowed": ("        if (!(rho[q] > rho[i] || (rho[q] == rho[i] && q < i))) continue;\n        const int64_t dq",
                            "        const int64_t dq"),
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
    lib.oracle_sapprox.argtypes = [vp, i64, i32, i64, i64, i64, vp, vp, vp, vp]
    return lib


def _golden_passes(lib):
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    for case in _cases():
        pts = np.ascontiguousarray(case["points"], dtype=np.int32)
        n, d = pts.shape
        rho = np.empty(n, np.int32)
        dep = np.empty(n, np.int32)
        d2 = np.empty(n, np.int64)
        pk = np.empty(n, np.int32)
        lib.oracle_sapprox(p(pts), n, d, case["d_cut"], case["eps_num"], case["eps_den"], p(rho), p(dep), p(d2), p(pk))
        if rho.tolist() != case["rho"] or dep.tolist() != case["dep"] or d2.tolist() != case["delta2"] \
                or pk.tolist() != case["pick"]:
            return False
    return True


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    assert not _golden_passes(_build(tmp_path, name, *MUTATIONS[name])), name


def test_subset_matches_full():
    ds = workloads.random_blobs(23, 1500, 3, 2500, blobs=5, spread=0.04, dup=7)
    rho, dep, d2, pk = oracle.sapprox(ds.points, 2500, 1, 2)
    idx = np.sort(np.random.default_rng(4).choice(1500, size=300, replace=False))
    sdep, sd2, spk = oracle.sapprox_dependent_subset(ds.points, rho, 2500, 1, 2, idx)
    np.testing.assert_array_equal(sdep, dep[idx])
    np.testing.assert_array_equal(sd2, d2[idx])
    np.testing.assert_array_equal(spk, pk[idx])


def test_unmutated_copy_passes(tmp_path):
    assert _golden_passes(_build(tmp_path, "identity", "int oracle_threads", "int oracle_threads"))
