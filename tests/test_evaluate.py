"""Rand index and decision-graph export (host-side), checked against a brute
force over all pairs and a hand-counted example."""
import itertools

import numpy as np
import pytest

from paper_2207_04649_gb300 import evaluate


def brute_rand(a, b):
    agree = total = 0
    for i, j in itertools.combinations(range(len(a)), 2):
        total += 1
        agree += (a[i] == a[j]) == (b[i] == b[j])
    return agree / total if total else 1.0


def test_hand_counted():
    # 4 points: a = {0,1}{2,3}, b = {0,1,2}{3}; 6 pairs: (0,1) same/same,
    # (0,2) diff/same, (0,3) diff/diff, (1,2) diff/same, (1,3) diff/diff,
    # (2,3) same/diff: 3 agree
    assert evaluate.rand_index([0, 0, 1, 1], [5, 5, 5, 7]) == pytest.approx(3 / 6)


@pytest.mark.parametrize("seed", range(6))
def test_against_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 60))
    a = rng.integers(-1, 4, size=n)
    b = rng.integers(-1, 5, size=n)
    assert evaluate.rand_index(a, b) == pytest.approx(brute_rand(a.tolist(), b.tolist()))


def test_identity_and_relabeling():
    a = np.array([3, 3, 7, -1, -1, 7, 9])
    assert evaluate.rand_index(a, a) == 1.0
    # renaming clusters changes nothing
    assert evaluate.rand_index(a, np.where(a == 3, 100, a)) == 1.0


def test_decision_graph_export(tmp_path):
    p = tmp_path / "dg.csv"
    r, d = evaluate.decision_graph([3, 1], [np.iinfo(np.int64).max, 16], str(p))
    assert r.tolist() == [3, 1]
    assert p.read_text().splitlines() == ["index,rho,delta2", f"0,3,{np.iinfo(np.int64).max}", "1,1,16"]
