"""Full-set parity on the workloads below 2M points: every point, not a sample.

The 1M x 8 set (exact DPC and S-Approx-DPC at eps 0.2) and all 256 problems
of the batched workload in one flush are compared with the oracle on every
element of rho, dep, delta2, the labels and the center count (Definitions
1-6; Section 5 for S-Approx-DPC). The oracle's complete outputs on these
sets take tens of minutes of host time, so ``tests/golden/full_parity.json``
holds SHA-256 digests of them, written by ``tests/golden/make_full_parity.py``
(which calls only the oracle and the input generators). Equal digests mean
equal arrays. When a digest differs, or the input or the oracle's source is
not the one recorded, the oracle runs here on the whole set and the arrays
are compared element by element, so a failure names the differing points.

A served-size job (2M x 8 with the served trace's recipe) runs in the served
mode beside small jobs; past 2M points parity is a seeded 20k-point sample
against the oracle's sampled forms plus properties on every point.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

I64MAX = np.iinfo(np.int64).max
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
GOLD = os.path.join(HERE, "golden", "full_parity.json")


@pytest.fixture(scope="module")
def dpc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2207_04649_gb300 as m
    m.lib()
    return m


def digest(a) -> str:
    a = np.ascontiguousarray(a)
    return hashlib.sha256(a.dtype.str.encode() + str(a.shape).encode() + a.tobytes()).hexdigest()


def input_digest(points, d_cut) -> str:
    return digest(np.ascontiguousarray(points, dtype=np.int32)) + f":{int(d_cut)}"


def stored(case):
    """The recorded digests of a case, or None when the file, the case or the
    oracle source it was made with is missing or different."""
    if not os.path.exists(GOLD):
        return None
    with open(GOLD) as f:
        g = json.load(f)
    with open(os.path.join(ROOT, "oracle", "dpc_oracle.c"), "rb") as f:
        if g.get("oracle_c_sha256") != hashlib.sha256(f.read()).hexdigest():
            return None
    return g.get("cases", {}).get(case)


def exact_oracle(points, d_cut, rho_min, delta_min):
    r = oracle.rho(points, d_cut)
    dep, d2 = oracle.dependent(points, r)
    lab, nc = oracle.label(r, dep, d2, rho_min, delta_min)
    return {"rho": r, "dep": dep, "delta2": d2, "label": lab, "n_centers": nc}


def sapprox_oracle(points, d_cut, num, den, rho_min, delta_min):
    r, dep, d2, pk = oracle.sapprox(points, d_cut, num, den)
    lab, nc = oracle.sapprox_label(r, dep, d2, pk, rho_min, delta_min)
    return {"rho": r, "dep": dep, "delta2": d2, "pick": pk.astype(np.uint8), "label": lab, "n_centers": nc}


def assert_same(got: dict, want_digests, points, d_cut, live):
    """Every array of ``got`` equals the oracle's: by digest when the recorded
    digests belong to this input, else (or on any difference) element by
    element against the oracle run here."""
    if want_digests is not None and want_digests["input"] == input_digest(points, d_cut):
        if all(digest(got[k]) == want_digests[k] for k in got if k != "n_centers") \
                and int(got["n_centers"]) == want_digests["n_centers"]:
            return "digest"
    want = live()
    for k in got:
        if k == "n_centers":
            assert int(got[k]) == int(want[k])
        else:
            np.testing.assert_array_equal(got[k], want[k], err_msg=k)
    if want_digests is not None and want_digests["input"] == input_digest(points, d_cut):
        raise AssertionError("the library agrees with the oracle run here but not with the recorded digests")
    return "live"


def assert_properties(points, d_cut, rho, dep, d2, lab, nc, rho_min, delta_min):
    """Properties that hold at any size (ranks from the GPU densities)."""
    n = len(rho)
    assert (int(rho.astype(np.int64).sum()) - n) % 2 == 0 and rho.min() >= 1
    order = oracle.rank_order(rho)
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    assert dep[order[0]] == -1 and d2[order[0]] == I64MAX and (dep == -1).sum() == 1
    nz = dep >= 0
    assert np.all(rank[dep[nz]] < rank[nz])
    P = points.astype(np.int64)
    np.testing.assert_array_equal(((P[nz] - P[dep[nz]]) ** 2).sum(axis=1), d2[nz])
    noise = rho < rho_min
    ctr = ~noise & (d2 >= delta_min * delta_min)
    np.testing.assert_array_equal(lab == -1, noise)
    assert nc == int(ctr.sum())
    olab, onc = oracle.label(rho, dep, d2, rho_min, delta_min)
    np.testing.assert_array_equal(lab, olab)
    assert nc == onc


def test_plain_1m_8d_every_point(dpc):
    """The 1M x 8 workload, exact DPC, compared on all 1,000,000 points."""
    ds = workloads.plain_1m_8d()
    pts = ds.points
    r = dpc.cluster(pts, ds.d_cut, ds.rho_min, ds.delta_min, device=0)
    got = {k: r[k] for k in ("rho", "dep", "delta2", "label", "n_centers")}
    assert_properties(pts, ds.d_cut, got["rho"], got["dep"], got["delta2"], got["label"], got["n_centers"],
                      ds.rho_min, ds.delta_min)
    assert_same(got, stored("plain_1m_8d"), pts, ds.d_cut,
                lambda: exact_oracle(pts, ds.d_cut, ds.rho_min, ds.delta_min))


def test_plain_1m_8d_sapprox_every_point(dpc):
    """S-Approx-DPC at eps 0.2 on the 1M x 8 workload, all points: densities
    of the picks (-1 elsewhere), links, picks, labels and centers."""
    ds = workloads.plain_1m_8d()
    pts = ds.points
    n = ds.n
    with dpc.Context(0) as ctx:
        rho = np.full(n, -7, np.int32)
        dep = np.full(n, -7, np.int32)
        d2 = np.full(n, -7, np.int64)
        pk = np.full(n, 7, np.uint8)
        h = ctx.sapprox(pts, ds.d_cut, (1, 5), rho, dep, d2, pk)
        lab = np.full(n, -7, np.int32)
        nc = h.label(ds.rho_min, ds.delta_min, lab)
        h.release()
    got = {"rho": rho, "dep": dep, "delta2": d2, "pick": pk, "label": lab, "n_centers": nc}
    assert_same(got, stored("plain_1m_8d_sapprox"), pts, ds.d_cut,
                lambda: sapprox_oracle(pts, ds.d_cut, 1, 5, ds.rho_min, ds.delta_min))


def test_batch_256_every_problem_in_one_flush(dpc):
    """All 256 problems of the batched workload submitted together and run as
    one batch; each against the oracle on every point."""
    probs = workloads.batch_256()
    gold = stored("batch_256")
    with dpc.Context(0, mode=0) as ctx:
        jobs = [dpc.Job(ds.points, ds.d_cut, [(ds.rho_min, ds.delta_min)]) for ds in probs]
        for j in jobs:
            ctx.submit(j)
        ctx.flush()
        for j in jobs:
            s, res = ctx.poll(j.ticket)
            assert s == dpc.DPC_OK and res.status == dpc.DPC_OK
    ways = []
    for b, (j, ds) in enumerate(zip(jobs, probs)):
        got = {"rho": j.rho, "dep": j.dep, "delta2": j.delta2, "label": j.label[0], "n_centers": j.n_centers[0]}
        want = gold["problems"][b] if gold is not None and len(gold["problems"]) == len(probs) else None
        ways.append(assert_same(got, want, ds.points, ds.d_cut,
                                lambda ds=ds: exact_oracle(ds.points, ds.d_cut, ds.rho_min, ds.delta_min)))
    assert len(ways) == 256


def test_served_job_of_trace_size(dpc):
    """A 2M x 8 request (the served trace's largest n and d) in the served
    mode, admitted beside small requests: a seeded 20k-point sample against
    the oracle's sampled forms, properties and labels on every point, and
    the small requests on every point."""
    big = workloads.served_problem(6, 2_000_000, 8)
    small = [workloads.random_blobs(600 + i, 3000 + 500 * i, 2 + i % 5, 700, blobs=3, spread=0.05, dup=4)
             for i in range(4)]
    with dpc.Context(0, mode=1, max_inflight=2) as ctx:
        jb = dpc.Job(big.points, big.d_cut, [(big.rho_min, big.delta_min), (1, 4 * big.d_cut)])
        js = [dpc.Job(s.points, s.d_cut, [(s.rho_min, s.delta_min)]) for s in small]
        ctx.submit(js[0])
        ctx.submit(jb)
        for j in js[1:]:
            ctx.submit(j)
        for j in [jb] + js:
            s, res = ctx.wait(j.ticket, 600000)
            assert s == dpc.DPC_OK and res.status == dpc.DPC_OK, dpc.dpc_last_error()
    for j, s in zip(js, small):
        got = {"rho": j.rho, "dep": j.dep, "delta2": j.delta2, "label": j.label[0], "n_centers": j.n_centers[0]}
        assert_same(got, None, s.points, s.d_cut,
                    lambda s=s: exact_oracle(s.points, s.d_cut, s.rho_min, s.delta_min))
    pts = big.points
    n = big.n
    idx = np.sort(np.random.default_rng(61).choice(n, size=20_000, replace=False))
    np.testing.assert_array_equal(jb.rho[idx], oracle.rho_subset(pts, big.d_cut, idx))
    sdep, sd2 = oracle.dependent_subset(pts, jb.rho, idx)
    np.testing.assert_array_equal(jb.dep[idx], sdep)
    np.testing.assert_array_equal(jb.delta2[idx], sd2)
    for q, (rmin, dmin) in enumerate([(big.rho_min, big.delta_min), (1, 4 * big.d_cut)]):
        assert_properties(pts, big.d_cut, jb.rho, jb.dep, jb.delta2, jb.label[q], jb.n_centers[q], rmin, dmin)
