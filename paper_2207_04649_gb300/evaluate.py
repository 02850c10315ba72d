"""Host-side evaluation helpers (no counterpart on the device path).

``rand_index`` is the accuracy measure the paper reports for its
approximation algorithms against Ex-DPC's labels (Section 5, "Quantitative
evaluation"): the share of point pairs on which two clusterings agree (both
put the pair in one cluster, or both split it). Noise points (label -1) form
one class of their own. It is computed exactly from the contingency table
with Python integers.

``decision_graph`` exports the data of the decision graph of Section 2.1
(Example 1): per point, its local density and dependent distance (squared,
INT64_MAX for the densest point), as arrays or a CSV file; plotting is left
to the caller.
"""
from __future__ import annotations

import numpy as np


def _pairs(counts: np.ndarray) -> int:
    c = counts.astype(object)
    return int(sum(x * (x - 1) // 2 for x in c))


def rand_index(labels_a, labels_b) -> float:
    """Rand index of two labelings of the same n points (1.0 when n < 2)."""
    a = np.asarray(labels_a, dtype=np.int64).ravel()
    b = np.asarray(labels_b, dtype=np.int64).ravel()
    if a.shape != b.shape:
        raise ValueError("labelings differ in length")
    n = a.size
    if n < 2:
        return 1.0
    _, ia = np.unique(a, return_inverse=True)
    _, ib = np.unique(b, return_inverse=True)
    joint = ia.astype(np.int64) * (int(ib.max()) + 1) + ib
    _, nij = np.unique(joint, return_counts=True)
    _, ai = np.unique(ia, return_counts=True)
    _, bj = np.unique(ib, return_counts=True)
    total = n * (n - 1) // 2
    same_both = _pairs(nij)
    agree = total + 2 * same_both - _pairs(ai) - _pairs(bj)
    return agree / total


def decision_graph(rho, delta2, path: str | None = None):
    """(rho, delta2) as int64 arrays; with ``path``, also a CSV file with the
    header ``index,rho,delta2``."""
    r = np.asarray(rho, dtype=np.int64).ravel()
    d = np.asarray(delta2, dtype=np.int64).ravel()
    if r.shape != d.shape:
        raise ValueError("rho and delta2 differ in length")
    if path is not None:
        with open(path, "w") as f:
            f.write("index,rho,delta2\n")
            for i, (x, y) in enumerate(zip(r.tolist(), d.tolist())):
                f.write(f"{i},{x},{y}\n")
    return r, d
