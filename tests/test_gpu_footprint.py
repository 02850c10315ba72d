"""The served mode's admission estimate against what a run really holds.

The served loop admits jobs while the sum of their estimated device bytes
(dpc_job_footprint) stays under hbm_cap_bytes. Each problem below is run
alone through the library, and the most device memory its batch held at
once (dpc_info.device_bytes_peak, counted in stream order) must not exceed
that estimate. The problems are drawn like the served trace's requests:
blob mixtures with 5 % noise in d = 2 .. 8, each with its own cutoff.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dpc():
    import paper_2207_04649_gb300 as dpc
    return dpc


def run_peak(dpc, ds, method):
    with dpc.Context(0) as ctx:
        if method == 2:
            h = ctx.sapprox(ds.points, ds.d_cut, 0.8)
        else:
            h = ctx.density(ds.points, ds.d_cut)
            if method == 1:
                h.dependent_approx()
            else:
                h.dependent()
        lab = np.empty(len(ds.points), np.int32)
        h.label(ds.rho_min, ds.delta_min, lab)
        peak = h.info()["device_bytes_peak"]
        h.release()
    return peak


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("n", [20_000, 200_000])
def test_exact_run_fits_its_estimate(dpc, n, d):
    ds = workloads.served_problem(seed=40 + d, n=n, d=d)
    peak = run_peak(dpc, ds, 0)
    est = dpc.dpc_job_footprint(n, d, 0)
    assert 0 < peak <= est, (n, d, peak, est)


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("d", [3, 8])
def test_approximate_runs_fit_their_estimate(dpc, d, method):
    n = 200_000
    ds = workloads.served_problem(seed=60 + d, n=n, d=d)
    peak = run_peak(dpc, ds, method)
    est = dpc.dpc_job_footprint(n, d, method)
    assert 0 < peak <= est, (n, d, method, peak, est)
