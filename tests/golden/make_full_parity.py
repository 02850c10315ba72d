"""Writes tests/golden/full_parity.json: SHA-256 digests of the oracle's
complete outputs on the full-size workloads that the GPU tests compare on
every point (the 1M x 8 set, exact and S-Approx-DPC at eps 0.2, and all 256
problems of the batched workload).

The digests are expected values written by this script, which calls only the
oracle (``oracle/``) and the seeded input generators (``workloads/``); the
GPU tests hash the library's outputs the same way and compare. Each case also
records the digest of its input points and of the oracle's C source, so a
test whose input or oracle differs from the one recorded here computes the
oracle's outputs itself instead of trusting the file.

Usage: python tests/golden/make_full_parity.py [case ...]   (about an hour
on 8 host cores for all cases).
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_parity.json")


def digest(a) -> str:
    """SHA-256 of an array's little-endian bytes in C order."""
    a = np.ascontiguousarray(a)
    return hashlib.sha256(a.dtype.str.encode() + str(a.shape).encode() + a.tobytes()).hexdigest()


def input_digest(points, d_cut) -> str:
    return digest(np.ascontiguousarray(points, dtype=np.int32)) + f":{int(d_cut)}"


def oracle_digest() -> str:
    with open(os.path.join(ROOT, "oracle", "dpc_oracle.c"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def exact_case(points, d_cut, rho_min, delta_min) -> dict:
    """Definitions 1-6 by the oracle's Scan (Section 2.2)."""
    r = oracle.rho(points, d_cut)
    dep, d2 = oracle.dependent(points, r)
    lab, nc = oracle.label(r, dep, d2, rho_min, delta_min)
    return {"input": input_digest(points, d_cut), "rho": digest(r), "dep": digest(dep), "delta2": digest(d2),
            "label": digest(lab), "n_centers": int(nc), "rho_sum": int(r.astype(np.int64).sum())}


def sapprox_case(points, d_cut, num, den, rho_min, delta_min) -> dict:
    """S-Approx-DPC (Section 5) by the oracle."""
    r, dep, d2, pk = oracle.sapprox(points, d_cut, num, den)
    lab, nc = oracle.sapprox_label(r, dep, d2, pk, rho_min, delta_min)
    return {"input": input_digest(points, d_cut), "eps": [num, den], "rho": digest(r), "dep": digest(dep),
            "delta2": digest(d2), "pick": digest(pk.astype(np.uint8)), "label": digest(lab),
            "n_centers": int(nc), "picks": int(pk.sum())}


def case_plain_1m_8d() -> dict:
    ds = workloads.plain_1m_8d()
    return exact_case(ds.points, ds.d_cut, ds.rho_min, ds.delta_min)


def case_plain_1m_8d_sapprox() -> dict:
    ds = workloads.plain_1m_8d()
    return sapprox_case(ds.points, ds.d_cut, 1, 5, ds.rho_min, ds.delta_min)


def case_batch_256() -> dict:
    return {"problems": [exact_case(ds.points, ds.d_cut, ds.rho_min, ds.delta_min)
                         for ds in workloads.batch_256()]}


CASES = {"plain_1m_8d": case_plain_1m_8d, "plain_1m_8d_sapprox": case_plain_1m_8d_sapprox,
         "batch_256": case_batch_256}


def main(names) -> None:
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    data["oracle_c_sha256"] = oracle_digest()
    data["digest"] = "sha256 of dtype string + shape string + little-endian C-order bytes"
    data.setdefault("cases", {})
    for name in names or list(CASES):
        t0 = time.time()
        data["cases"][name] = CASES[name]()
        print(f"{name}: {time.time() - t0:.0f} s on {oracle.threads()} threads", flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
