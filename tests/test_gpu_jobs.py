"""Batched and served jobs: every dataset's result in a batch or in the
served mix is the same bits as the dataset run alone, and as the oracle."""
import threading

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dpc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2207_04649_gb300 as m
    m.lib()
    return m


def small_problems(seed=40, count=14):
    """Uneven n, d and d_cut in one batch (d 1..8, some tiny and empty)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice([0, 1, 7, 150, 900, 2500, 4000]))
        d = int(rng.integers(1, 9))
        dc = int(rng.choice([60, 400, 1500, 6000]))
        ds = workloads.random_blobs(seed * 100 + i, n, d, dc, blobs=int(rng.integers(1, 6)),
                                    spread=float(rng.choice([0.01, 0.05, 0.2])), dup=3 if n > 10 else 0)
        qs = [(2, dc + 1), (1, 4 * dc), (int(rng.integers(1, 6)), 10 * dc)][: 1 + i % 3]
        out.append((ds.points, dc, qs))
    return out


def expected(points, dc, qs):
    r = oracle.rho(points, dc)
    dep, d2 = oracle.dependent(points, r)
    labs = [oracle.label(r, dep, d2, a, b) for a, b in qs]
    return r, dep, d2, labs


def check_job(job, points, dc, qs):
    r, dep, d2, labs = expected(points, dc, qs)
    np.testing.assert_array_equal(job.rho, r)
    np.testing.assert_array_equal(job.dep, dep)
    np.testing.assert_array_equal(job.delta2, d2)
    for q, (lab, nc) in enumerate(labs):
        np.testing.assert_array_equal(job.label[q], lab)
        assert job.n_centers[q] == nc


def test_batched_flush_matches_oracle(dpc):
    probs = small_problems()
    with dpc.Context(0, mode=0) as ctx:
        jobs = [dpc.Job(p, dc, qs) for p, dc, qs in probs]
        for j in jobs:
            ctx.submit(j)
        ctx.flush()
        for j, (p, dc, qs) in zip(jobs, probs):
            s, res = ctx.poll(j.ticket)
            assert s == dpc.DPC_OK and res.status == dpc.DPC_OK
            check_job(j, p, dc, qs)


@pytest.mark.parametrize("knobs", [dict(bf_rank=0), dict(bf_rank=1 << 30)], ids=["tree_only", "brute_force_only"])
def test_batched_open_point_passes(dpc, knobs):
    """A batch of uneven datasets whose open points all go through the tree
    search (bf_rank 0) or all through the brute force over the rank prefix."""
    probs = small_problems(seed=42, count=16)
    with dpc.Context(0, mode=0) as ctx:
        ctx.tune(**knobs)
        jobs = [dpc.Job(p, dc, qs) for p, dc, qs in probs]
        for j in jobs:
            ctx.submit(j)
        ctx.flush()
        for j, (p, dc, qs) in zip(jobs, probs):
            s, res = ctx.poll(j.ticket)
            assert s == dpc.DPC_OK and res.status == dpc.DPC_OK
            check_job(j, p, dc, qs)


def expected_method(method, points, dc, qs, eps):
    """The oracle's rho, dep, delta2, aux and labels for one job."""
    if method == "sapprox":
        r, dep, d2, pk = oracle.sapprox(points, dc, *eps)
        return r, dep, d2, pk, [oracle.sapprox_label(r, dep, d2, pk, a, b) for a, b in qs]
    r = oracle.rho(points, dc)
    if method == "approx":
        dep, d2, ex = oracle.approx_dependent(points, r, dc)
    else:
        dep, d2 = oracle.dependent(points, r)
        ex = None
    return r, dep, d2, ex, [oracle.label(r, dep, d2, a, b) for a, b in qs]


def check_method_job(job, method, points, dc, qs, eps):
    r, dep, d2, aux, labs = expected_method(method, points, dc, qs, eps)
    np.testing.assert_array_equal(job.rho, r)
    np.testing.assert_array_equal(job.dep, dep)
    np.testing.assert_array_equal(job.delta2, d2)
    if aux is not None:
        np.testing.assert_array_equal(job.aux.astype(bool), aux)
    for q, (lab, nc) in enumerate(labs):
        np.testing.assert_array_equal(job.label[q], lab)
        assert job.n_centers[q] == nc


METHOD_CYCLE = ["approx", "sapprox", "sapprox", "exact", "approx", "approx", "sapprox"]
EPS_CYCLE = [(4, 5), (1, 5), (1, 1), (3, 1)]


@pytest.mark.parametrize("mode", [0, 1])
def test_jobs_of_every_method(dpc, mode):
    """Approx-DPC, S-Approx-DPC and exact jobs mixed in one submission (runs
    of one method become batches; uneven n, d 1..8, some empty), each job
    against the oracle of its method."""
    probs = small_problems(seed=43, count=21)
    with dpc.Context(0, mode=mode, max_inflight=2) as ctx:
        jobs = []
        for i, (p, dc, qs) in enumerate(probs):
            m = METHOD_CYCLE[i % len(METHOD_CYCLE)]
            eps = EPS_CYCLE[i % len(EPS_CYCLE)]
            j = dpc.Job(p, dc, qs, method=m, eps=eps)
            jobs.append((j, m, eps))
            ctx.submit(j)
        if mode == 0:
            ctx.flush()
        for (j, m, eps), (p, dc, qs) in zip(jobs, probs):
            s, res = ctx.wait(j.ticket, 120000)
            assert s == dpc.DPC_OK and res.status == dpc.DPC_OK, (m, res.status)
            check_method_job(j, m, p, dc, qs, eps)


def test_approx_keys_wider_than_64_bits(dpc):
    """Approx-DPC on an 8-d set whose grid keys need more than one word."""
    rng = np.random.default_rng(72)
    pts = rng.integers(0, 1 << 29, size=(2500, 8)).astype(np.int32)
    pts[800:1300] = pts[:500] + rng.integers(-3, 4, size=(500, 8)).astype(np.int32)
    pts = np.clip(pts, 0, (1 << 30) - 1)
    dc = 40
    with dpc.Context(0) as ctx:
        h = ctx.density(pts, dc)
        dep = np.empty(len(pts), np.int32)
        d2 = np.empty(len(pts), np.int64)
        ex = np.empty(len(pts), np.uint8)
        h.dependent_approx(dep, d2, ex)
        h.release()
    r = oracle.rho(pts, dc)
    odep, od2, oex = oracle.approx_dependent(pts, r, dc)
    np.testing.assert_array_equal(dep, odep)
    np.testing.assert_array_equal(d2, od2)
    np.testing.assert_array_equal(ex.astype(bool), oex)


def test_batch_equals_alone_on_blob_workload(dpc):
    """A slice of the 256-problem batch: bits equal to each problem alone."""
    probs = workloads.batch_256(count=12)
    with dpc.Context(0, mode=0) as ctx:
        jobs = [dpc.Job(ds.points, ds.d_cut, [(ds.rho_min, ds.delta_min)]) for ds in probs]
        for j in jobs:
            ctx.submit(j)
        ctx.flush()
    for j, ds in zip(jobs, probs):
        alone = dpc.cluster(ds.points, ds.d_cut, ds.rho_min, ds.delta_min)
        np.testing.assert_array_equal(j.rho, alone["rho"])
        np.testing.assert_array_equal(j.dep, alone["dep"])
        np.testing.assert_array_equal(j.delta2, alone["delta2"])
        np.testing.assert_array_equal(j.label[0], alone["label"])
        assert j.n_centers[0] == alone["n_centers"]
    # and the smallest ones against the oracle
    for j, ds in sorted(zip(jobs, probs), key=lambda t: t[1].n)[:3]:
        check_job(j, ds.points, ds.d_cut, [(ds.rho_min, ds.delta_min)])


def test_served_mode_concurrent_submitters(dpc):
    probs = small_problems(seed=41, count=20)
    with dpc.Context(0, mode=1, max_inflight=3) as ctx:
        jobs = [dpc.Job(p, dc, qs) for p, dc, qs in probs]
        lock = threading.Lock()

        def submit(chunk):
            for j in chunk:
                with lock:
                    pass
                ctx.submit(j)

        threads = [threading.Thread(target=submit, args=(jobs[i::4],)) for i in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        for j in jobs:
            s, res = ctx.wait(j.ticket, 120000)
            assert s == dpc.DPC_OK, dpc.dpc_last_error()
            assert res.run_ms >= 0.0 and res.queue_ms >= 0.0
    for j, (p, dc, qs) in zip(jobs, probs):
        check_job(j, p, dc, qs)


def test_served_admission_under_small_cap(dpc):
    """A cap that fits about one job at a time still finishes every job;
    a job that can never fit is refused at submit."""
    probs = small_problems(seed=42, count=6)
    cap = max(dpc.dpc_job_footprint(len(p), p.shape[1] if p.ndim == 2 and p.size else 1, 0) for p, _, _ in probs) + (4 << 20)
    with dpc.Context(0, mode=1, hbm_cap_bytes=cap, max_inflight=2) as ctx:
        jobs = [dpc.Job(p, dc, qs) for p, dc, qs in probs]
        for j in jobs:
            ctx.submit(j)
        for j in jobs:
            s, _ = ctx.wait(j.ticket, 120000)
            assert s == dpc.DPC_OK
        big = dpc.Job(np.zeros((2_000_000, 8), np.int32), 10, [(1, 11)])
        with pytest.raises(dpc.DpcError) as e:
            ctx.submit(big)
        assert e.value.status == dpc.DPC_ERR_CAPACITY
    for j, (p, dc, qs) in zip(jobs, probs):
        check_job(j, p, dc, qs)


def test_poll_unknown_ticket_and_wait_timeout(dpc):
    with dpc.Context(0, mode=0) as ctx:
        s, _ = ctx.poll(987654)
        assert s == dpc.DPC_ERR_STATE
        j = dpc.Job(np.zeros((10, 2), np.int32), 5, [(1, 6)])
        ctx.submit(j)
        s, _ = ctx.poll(j.ticket)
        assert s == dpc.DPC_PENDING          # batched mode: nothing runs before flush
        s, _ = ctx.wait(j.ticket, 10)
        assert s == dpc.DPC_ERR_TIMEOUT
        ctx.flush()
        s, _ = ctx.poll(j.ticket)
        assert s == dpc.DPC_OK


def test_device_jobs_match_host_jobs(dpc):
    """Jobs whose points and outputs live in device memory give the same bits
    as host-memory jobs, in one batch mixed with host jobs."""
    import torch
    probs = small_problems(seed=43, count=10)
    with dpc.Context(0, mode=0, profiling=True) as ctx:
        dev = [dpc.Job(torch.from_numpy(np.ascontiguousarray(p)).cuda(), dc, qs) for p, dc, qs in probs]
        host = [dpc.Job(p, dc, qs) for p, dc, qs in probs]
        torch.cuda.synchronize()
        for a, b in zip(dev, host):
            ctx.submit(a)
            ctx.submit(b)
        ctx.flush()
        for j in dev + host:
            s, _ = ctx.poll(j.ticket)
            assert s == dpc.DPC_OK
        info = ctx.last_batch_info()
        assert info["n"] == 2 * sum(p.shape[0] for p, _, _ in probs)
        assert info["cand_pairs"] > 0 and info["ms_rho"] > 0.0
    for a, b in zip(dev, host):
        np.testing.assert_array_equal(a.rho.cpu().numpy(), b.rho)
        np.testing.assert_array_equal(a.dep.cpu().numpy(), b.dep)
        np.testing.assert_array_equal(a.delta2.cpu().numpy(), b.delta2)
        np.testing.assert_array_equal(a.label.cpu().numpy(), b.label)
        np.testing.assert_array_equal(a.n_centers, b.n_centers)
    for b, (p, dc, qs) in zip(host, probs):
        check_job(b, p, dc, qs)


def test_page_locked_host_jobs(dpc):
    """Host jobs in page-locked memory (points, outputs or both), which a
    batch reads and writes from the device directly, mixed with pageable
    host jobs and device jobs: the oracle's bits for every job."""
    import torch
    probs = small_problems(seed=47, count=12)
    jobs = []
    with dpc.Context(0, mode=0) as ctx:
        for i, (p, dc, qs) in enumerate(probs):
            kind = i % 4
            if kind == 0:    # pinned points and outputs
                j = dpc.Job(torch.from_numpy(np.ascontiguousarray(p)).pin_memory().numpy(), dc, qs, pinned=True)
            elif kind == 1:  # pinned points, pageable outputs
                j = dpc.Job(torch.from_numpy(np.ascontiguousarray(p)).pin_memory().numpy(), dc, qs)
            elif kind == 2:  # pageable points, pinned outputs
                j = dpc.Job(p, dc, qs, pinned=True)
            else:
                j = dpc.Job(torch.from_numpy(np.ascontiguousarray(p)).cuda(), dc, qs)
            jobs.append(j)
        torch.cuda.synchronize()
        for j in jobs:
            ctx.submit(j)
        ctx.flush()
        for j in jobs:
            assert ctx.poll(j.ticket)[0] == dpc.DPC_OK
    for j, (p, dc, qs) in zip(jobs, probs):
        if j.is_device:
            for name in ("rho", "dep", "delta2", "label"):
                setattr(j, name, getattr(j, name).cpu().numpy())
        check_job(j, p, dc, qs)


def test_served_one_job_per_batch(dpc):
    """max_batch_jobs = 1 serves the jobs one at a time with the same results."""
    probs = small_problems(seed=44, count=6)
    with dpc.Context(0, mode=1, max_inflight=1) as ctx:
        ctx.tune(max_batch_jobs=1)
        assert ctx.tuning("max_batch_jobs") == 1
        jobs = [dpc.Job(p, dc, qs) for p, dc, qs in probs]
        for j in jobs:
            ctx.submit(j)
        for j in jobs:
            s, _ = ctx.wait(j.ticket, 120000)
            assert s == dpc.DPC_OK
    for j, (p, dc, qs) in zip(jobs, probs):
        check_job(j, p, dc, qs)


def test_last_batch_info_before_any_batch(dpc):
    with dpc.Context(0, mode=0) as ctx:
        with pytest.raises(dpc.DpcError) as e:
            ctx.last_batch_info()
        assert e.value.status == dpc.DPC_ERR_STATE


def test_autotune_keeps_results_and_writes_cache(dpc, tmp_path):
    probs = workloads.batch_256(count=16)
    cache = str(tmp_path / "tune.txt")
    with dpc.Context(0, mode=0) as ctx:
        ref = [dpc.Job(ds.points, ds.d_cut, [(ds.rho_min, ds.delta_min)]) for ds in probs]
        for j in ref:
            ctx.submit(j)
        ctx.flush()
        for j in ref:
            assert ctx.poll(j.ticket)[0] == dpc.DPC_OK
    with dpc.Context(0, mode=0, tune_cache=cache) as ctx:
        jobs = [dpc.Job(ds.points, ds.d_cut, [(ds.rho_min, ds.delta_min)]) for ds in probs]
        rep = ctx.autotune(jobs, repeats=1)
        assert "kch=" in rep and "dmax=" in rep
        for k in ("kch", "qch", "bf_rank"):
            assert f"{k}={ctx.tuning(k)}" in rep
        with pytest.raises(dpc.DpcError):
            ctx.autotune(jobs, repeats=0)
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and lines[0].startswith("dmax=")
    for a, b in zip(jobs, ref):
        np.testing.assert_array_equal(a.rho, b.rho)
        np.testing.assert_array_equal(a.dep, b.dep)
        np.testing.assert_array_equal(a.delta2, b.delta2)
        np.testing.assert_array_equal(a.label, b.label)
    # a new context reads the cache and runs the same batch with its entry
    with dpc.Context(0, mode=0, tune_cache=cache) as ctx:
        again = [dpc.Job(ds.points, ds.d_cut, [(ds.rho_min, ds.delta_min)]) for ds in probs]
        for j in again:
            ctx.submit(j)
        ctx.flush()
        for j in again:
            assert ctx.poll(j.ticket)[0] == dpc.DPC_OK
    for a, b in zip(again, ref):
        np.testing.assert_array_equal(a.label, b.label)
        np.testing.assert_array_equal(a.dep, b.dep)


@pytest.mark.parametrize("mode", [0, 1])
def test_kept_jobs_answer_requeries_after_they_return(dpc, mode):
    """Jobs submitted with keep stay on the device after they finish: new
    (rho_min, delta_min) queries on the returned dataset (labels only, the
    decision-graph workflow of Section 2.1) give the oracle's labels, for
    every job of a batch; releasing them frees their share of the cap."""
    probs = small_problems(seed=45, count=8)
    with dpc.Context(0, mode=mode, max_inflight=2) as ctx:
        jobs = [dpc.Job(p, dc, qs, keep=(i % 3 != 2)) for i, (p, dc, qs) in enumerate(probs)]
        for j in jobs:
            ctx.submit(j)
        if mode == 0:
            ctx.flush()
        for j in jobs:
            s, res = ctx.wait(j.ticket, 120000)
            assert s == dpc.DPC_OK
            assert (j.dataset is not None) == bool(j.c.keep)
        for j, (p, dc, qs) in zip(jobs, probs):
            check_job(j, p, dc, qs)
            if j.dataset is None:
                continue
            r, dep, d2, _ = expected(p, dc, qs)
            for rmin, dmin in [(1, dc + 1), (3, 2 * dc + 7), (max(1, int(r.max()) if len(r) else 1), 50 * dc)]:
                lab = np.full(len(p), -7, np.int32)
                nc = j.dataset.label(rmin, dmin, lab)
                olab, onc = oracle.label(r, dep, d2, rmin, dmin)
                np.testing.assert_array_equal(lab, olab)
                assert nc == onc
            assert j.dataset.info()["n"] == len(p)
        for j in jobs:
            if j.dataset is not None:
                j.dataset.release()


def test_kept_dataset_holds_its_bytes_until_released(dpc):
    """A kept dataset counts against the served cap: with a cap that fits
    one job, a second job is admitted only after the first one's dataset is
    released."""
    import time
    p = workloads.random_blobs(71, 20000, 3, 900, blobs=4, spread=0.05).points
    q = [(2, 2000)]
    cap = dpc.dpc_job_footprint(20000, 3, 0) * 3 // 2  # one job's reservation fits, two do not
    with dpc.Context(0, mode=1, hbm_cap_bytes=cap, max_inflight=1) as ctx:
        a = dpc.Job(p, 900, q, keep=True)
        ctx.submit(a)
        assert ctx.wait(a.ticket, 60000)[0] == dpc.DPC_OK
        b = dpc.Job(p, 900, q)
        ctx.submit(b)
        time.sleep(0.5)
        assert ctx.poll(b.ticket)[0] == dpc.DPC_PENDING  # held back by a's dataset
        a.dataset.release()
        assert ctx.wait(b.ticket, 60000)[0] == dpc.DPC_OK
    np.testing.assert_array_equal(a.label, b.label)


def test_small_job_is_not_held_back_by_a_large_one(dpc):
    """Served: a 2M x 8 request followed by a small one; the points cap puts
    them in separate batches on separate workers, so the small one finishes
    first, with the oracle's bits."""
    big = workloads.served_problem(7, 2_000_000, 8)
    small = workloads.random_blobs(72, 3000, 3, 700, blobs=3, spread=0.05, dup=4)
    with dpc.Context(0, mode=1, max_inflight=2) as ctx:
        assert ctx.tuning("max_batch_points") == 1 << 20
        jb = dpc.Job(big.points, big.d_cut, [(big.rho_min, big.delta_min)])
        js = dpc.Job(small.points, small.d_cut, [(small.rho_min, small.delta_min)])
        ctx.submit(jb)
        ctx.submit(js)
        s_small, r_small = ctx.wait(js.ticket, 600000)
        assert s_small == dpc.DPC_OK
        s_big, r_big = ctx.wait(jb.ticket, 600000)
        assert s_big == dpc.DPC_OK
        done_small = r_small.queue_ms + r_small.run_ms
        done_big = r_big.queue_ms + r_big.run_ms
        assert done_small < done_big, (done_small, done_big)
    check_job(js, small.points, small.d_cut, [(small.rho_min, small.delta_min)])


def test_one_query_job_finishes_before_four_query_job_of_its_batch(dpc):
    """In one batch, a job is done as soon as its own outputs are written."""
    probs = small_problems(seed=46, count=2)
    p0, dc0, _ = probs[0]
    p1, dc1, _ = probs[1]
    with dpc.Context(0, mode=0) as ctx:
        a = dpc.Job(p0, dc0, [(2, dc0 + 1)])
        b = dpc.Job(p1, dc1, [(2, dc1 + 1), (1, 2 * dc1), (3, 3 * dc1), (1, 9 * dc1)])
        ctx.submit(a)
        ctx.submit(b)
        ctx.flush()
        _, ra = ctx.poll(a.ticket)
        _, rb = ctx.poll(b.ticket)
        assert ra.status == rb.status == dpc.DPC_OK
        assert ra.run_ms <= rb.run_ms
    check_job(a, p0, dc0, [(2, dc0 + 1)])
    check_job(b, p1, dc1, [(2, dc1 + 1), (1, 2 * dc1), (3, 3 * dc1), (1, 9 * dc1)])
