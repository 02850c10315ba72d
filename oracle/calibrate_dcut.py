"""Calibrate the cutoff distance of the large named workloads.

Test infrastructure (part of the oracle). For each workload it draws the
seeded points from ``workloads``, takes a seeded sample of points, computes
their exact local density against all n points with the oracle
(Definition 1), and bisects the integer d_cut until the sample's mean local
density is as close as possible to the workload's target. The result is
frozen in ``workloads/calibrated.json`` so every run uses the same d_cut.

    python -m oracle.calibrate_dcut
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
import workloads  # noqa: E402

TARGETS = {
    # name: (draw function, seed, n, target mean rho, sample size)
    "plain_5p8m_3d": (workloads._c2_draw, 2, 5_800_000, 100.0, 1000),
    "plain_1m_8d": (workloads._c3_draw, 3, 1_000_000, 50.0, 2000),
}


def calibrate(name: str) -> dict:
    draw, seed, n, target, m = TARGETS[name]
    pts = draw(seed, n)[0]
    idx = np.random.default_rng(1000 + seed).choice(n, size=m, replace=False)

    def mean_rho(dc: int) -> float:
        return float(oracle.rho_subset(pts, dc, idx).mean())

    lo, hi = 1, 2
    while mean_rho(hi) < target:
        lo, hi = hi, hi * 2
    # invariant: mean_rho(lo) < target <= mean_rho(hi)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if mean_rho(mid) < target:
            lo = mid
        else:
            hi = mid
    best = min((lo, hi), key=lambda dc: abs(mean_rho(dc) - target))
    return {"seed": seed, "n": n, "d_cut": int(best), "target_mean_rho": target,
            "sample_mean_rho": mean_rho(best), "sample_size": m,
            "sample_seed": 1000 + seed}


def main() -> None:
    out_path = os.path.join(os.path.dirname(workloads.__file__), "calibrated.json")
    res = {}
    for name in TARGETS:
        t = time.time()
        res[name] = calibrate(name)
        print(name, res[name], f"{time.time() - t:.1f}s", flush=True)
    with open(out_path, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
