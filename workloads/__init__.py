"""Seeded synthetic inputs for exact Density-Peaks Clustering.

This module only draws points and parameters. It holds none of the
clustering arithmetic, so both the CUDA path and the CPU oracle can take
their inputs from it without sharing any of the method.

The paper evaluates on Airline (5,810,462 x 3), Household, PAMAP2 and Sensor
(928,991 x 8) (Section 5, "Datasets"); none of them is available here. The
workloads below are synthetic stand-ins of the same shape: integer
coordinates in [0, 100000], Gaussian-blob mixtures with skewed weights and
uniform noise. Every draw is seeded with numpy's PCG64 generator.

Cutoff distances: the named plain workloads take d_cut from
``calibrated.json`` (written by ``oracle/calibrate_dcut.py`` so that the mean
local density hits its target on a seeded sample). The batched and served
workloads use ``dcut_for_mean_rho``, a closed-form estimate from the mixture
parameters (expected neighbours of a point drawn from a Gaussian mixture),
so no clustering arithmetic is run to make them.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

DOMAIN = 100_000
_HERE = os.path.dirname(os.path.abspath(__file__))
_CALIBRATED = os.path.join(_HERE, "calibrated.json")


@dataclass
class Dataset:
    """One clustering problem: int32 points (n x d) and its parameters."""
    name: str
    points: np.ndarray
    d_cut: int
    rho_min: int
    delta_min: int
    queries: list = field(default_factory=list)  # extra (rho_min, delta_min) re-queries
    arrival_s: float = 0.0
    seed: int = 0

    @property
    def n(self) -> int:
        return int(self.points.shape[0])

    @property
    def d(self) -> int:
        return int(self.points.shape[1])


def _finish(rng, pts) -> np.ndarray:
    """Round to the integer lattice, clip to the domain, shuffle the order."""
    pts = np.clip(np.rint(pts), 0, DOMAIN).astype(np.int32)
    return np.ascontiguousarray(pts[rng.permutation(pts.shape[0])])


def _counts(rng, n_total, weights, noise_frac):
    n_noise = int(round(noise_frac * n_total))
    w = np.asarray(weights, dtype=np.float64)
    blob = rng.multinomial(n_total - n_noise, w / w.sum())
    return blob, n_noise


def isotropic_mixture(rng, n, d, centers, sigmas, weights, noise_frac) -> np.ndarray:
    """Gaussian blobs N(center_b, sigma_b^2 I) plus uniform noise in the domain."""
    blob, n_noise = _counts(rng, n, weights, noise_frac)
    parts = [centers[b] + sigmas[b] * rng.standard_normal((blob[b], d)) for b in range(len(blob))]
    parts.append(rng.uniform(0, DOMAIN, size=(n_noise, d)))
    return _finish(rng, np.concatenate(parts, axis=0))


def anisotropic_mixture(rng, n, d, centers, eigvals, weights, noise_frac) -> np.ndarray:
    """Gaussian blobs with covariance Q diag(eigvals_b) Q^T (Q a random
    orthogonal matrix from the QR factors of a Gaussian matrix)."""
    blob, n_noise = _counts(rng, n, weights, noise_frac)
    parts = []
    for b in range(len(blob)):
        q, r = np.linalg.qr(rng.standard_normal((d, d)))
        q = q * np.sign(np.diag(r))
        z = rng.standard_normal((blob[b], d)) * np.sqrt(eigvals[b])
        parts.append(centers[b] + z @ q.T)
    parts.append(rng.uniform(0, DOMAIN, size=(n_noise, d)))
    return _finish(rng, np.concatenate(parts, axis=0))


def _ball_volume(d: int) -> float:
    return math.pi ** (d / 2) / math.gamma(d / 2 + 1)


def dcut_for_mean_rho(n, d, weights, log_det_cov, noise_frac, target) -> int:
    """Closed-form cutoff so that the mean local density is about ``target``.

    A point drawn from blob b sees blob b's density with mean
    (4 pi)^(-d/2) det(Sigma_b)^(-1/2); with mixture weights pi_b the expected
    number of other points within r is about
    n * V_d r^d * sum_b pi_b^2 (4 pi)^(-d/2) det(Sigma_b)^(-1/2) (+ the noise
    term). Solving for r gives the estimate (clipping at the domain edge and
    blob overlap are ignored)."""
    w = np.asarray(weights, dtype=np.float64)
    pi = (1.0 - noise_frac) * w / w.sum()
    k = float(np.sum(pi ** 2 * (4 * math.pi) ** (-d / 2) * np.exp(-0.5 * np.asarray(log_det_cov))))
    k += noise_frac ** 2 / float(DOMAIN) ** d
    r = ((max(target - 1.0, 0.5)) / (n * _ball_volume(d) * k)) ** (1.0 / d)
    return max(1, int(round(r)))


def _zipf_weights(k, s):
    return np.arange(1, k + 1, dtype=np.float64) ** (-s)


def _load_calibrated() -> dict:
    if not os.path.exists(_CALIBRATED):
        return {}
    with open(_CALIBRATED) as f:
        return json.load(f)


# ------------------------------------------------------------------ named workloads

def plain_20k_2d(seed: int = 1) -> Dataset:
    """n=20,000, d=2: 10 isotropic blobs (sigma 2000, centers in
    [10000, 90000]^2) + 5% uniform noise; d_cut 1000, rho_min 5, delta_min 5000."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(10_000, 90_000, size=(10, 2))
    pts = isotropic_mixture(rng, 20_000, 2, centers, np.full(10, 2000.0), np.ones(10), 0.05)
    return Dataset("plain_20k_2d", pts, 1000, 5, 5000, seed=seed)


def _c2_draw(seed: int, n: int):
    rng = np.random.default_rng(seed)
    centers = rng.uniform(10_000, 90_000, size=(50, 3))
    sig = np.exp(rng.uniform(math.log(500), math.log(5000), size=50))
    w = _zipf_weights(50, 1.1)
    pts = isotropic_mixture(rng, n, 3, centers, sig, w, 0.02)
    return pts, w, sig


def plain_5p8m_3d(seed: int = 2, n: int = 5_800_000) -> Dataset:
    """n=5.8M, d=3 (stands in for Airline): 50 isotropic blobs with sigma
    log-uniform in [500, 5000] and Zipf(1.1) weights + 2% uniform noise;
    d_cut for mean rho ~ 100; rho_min 10, delta_min 10 d_cut."""
    pts, w, sig = _c2_draw(seed, n)
    cal = _load_calibrated().get("plain_5p8m_3d")
    if cal is not None and cal["seed"] == seed and cal["n"] == n:
        d_cut = int(cal["d_cut"])
    else:
        d_cut = dcut_for_mean_rho(n, 3, w, 3 * np.log(sig ** 2), 0.02, 100.0)
    return Dataset("plain_5p8m_3d", pts, d_cut, 10, 10 * d_cut, seed=seed)


def plain_2m_3d(seed: int = 2, n: int = 2_000_000) -> Dataset:
    """A 2M-point draw of the same 3-d mixture (the profiling case: its
    device footprint stays well under the bench case's); d_cut is the
    5.8M set's calibrated cutoff scaled by (5.8M / n)^(1/3), which keeps the
    expected neighbour count, and rho_min / delta_min follow it."""
    big = _load_calibrated().get("plain_5p8m_3d")
    base = int(big["d_cut"]) if big is not None else 178
    d_cut = int(round(base * (5_800_000 / n) ** (1.0 / 3.0)))
    pts, _, _ = _c2_draw(seed, n)
    return Dataset("plain_2m_3d", pts, d_cut, 10, 10 * d_cut, seed=seed)


def plain_5p8m_3d_dense(seed: int = 2, n: int = 5_800_000) -> Dataset:
    """The 5.8M x 3 set with a cutoff 4 times larger (mean rho about 64
    times larger, several thousand): the dense regime in which S-Approx-DPC's
    cells of G' hold many points each, as on the paper's data sets;
    rho_min and delta_min scale with it."""
    base = plain_5p8m_3d(seed, n)
    d_cut = 4 * base.d_cut
    return Dataset("plain_5p8m_3d_dense", base.points, d_cut, 640, 10 * d_cut, seed=seed)


def _c3_draw(seed: int, n: int):
    rng = np.random.default_rng(seed)
    centers = rng.uniform(10_000, 90_000, size=(20, 8))
    eig = np.exp(rng.uniform(math.log(1e6), math.log(1e8), size=(20, 8)))
    w = np.ones(20)
    pts = anisotropic_mixture(rng, n, 8, centers, eig, w, 0.0)
    return pts, w, eig


def plain_1m_8d(seed: int = 3, n: int = 1_000_000) -> Dataset:
    """n=1M, d=8 (stands in for Sensor): 20 anisotropic blobs, covariance
    eigenvalues log-uniform in [1e6, 1e8], clipped to the domain; d_cut for
    mean rho ~ 50; rho_min 5, delta_min 8 d_cut."""
    pts, w, eig = _c3_draw(seed, n)
    cal = _load_calibrated().get("plain_1m_8d")
    if cal is not None and cal["seed"] == seed and cal["n"] == n:
        d_cut = int(cal["d_cut"])
    else:
        d_cut = dcut_for_mean_rho(n, 8, w, np.log(eig).sum(axis=1), 0.0, 50.0)
    return Dataset("plain_1m_8d", pts, d_cut, 5, 8 * d_cut, seed=seed)


def plain_400k_8d(seed: int = 3, n: int = 400_000) -> Dataset:
    """A 400k-point draw of the same 8-d mixture (a profiling case well
    under the 1M set's footprint); d_cut is the 1M set's calibrated cutoff
    scaled by (1M / n)^(1/8), which keeps the expected neighbour count."""
    big = _load_calibrated().get("plain_1m_8d")
    base = int(big["d_cut"]) if big is not None else 4040
    d_cut = int(round(base * (1_000_000 / n) ** (1.0 / 8.0)))
    pts, _, _ = _c3_draw(seed, n)
    return Dataset("plain_400k_8d", pts, d_cut, 5, 8 * d_cut, seed=seed)


def _random_problem(rng, name, n, d, target_rho, noise_frac=0.05):
    """A blob mixture (5-30 blobs) + uniform noise with its own cutoff."""
    nb = int(rng.integers(5, 31))
    centers = rng.uniform(10_000, 90_000, size=(nb, d))
    sig = np.exp(rng.uniform(math.log(500), math.log(5000), size=nb))
    w = rng.uniform(0.2, 1.0, size=nb)
    pts = isotropic_mixture(rng, n, d, centers, sig, w, noise_frac)
    d_cut = dcut_for_mean_rho(n, d, w, d * np.log(sig ** 2), noise_frac, target_rho)
    rho_min = max(2, int(0.1 * target_rho))
    delta_min = int(round(rng.uniform(5, 10) * d_cut))
    return Dataset(name, pts, d_cut, rho_min, max(delta_min, d_cut + 1))


def batch_256(seed: int = 4, count: int = 256) -> list:
    """256 independent problems: n log-uniform on [1k, 200k], d in {2,3,4},
    blob mixtures + 5% noise, each with its own d_cut (mean rho 20-200),
    rho_min and delta_min."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(round(math.exp(rng.uniform(math.log(1_000), math.log(200_000)))))
        d = int(rng.integers(2, 5))
        target = float(rng.uniform(20, 200))
        ds = _random_problem(rng, f"batch_{b}", n, d, target)
        ds.seed = seed
        out.append(ds)
    return out


def served_trace(seed: int = 5, jobs: int = 2000, rate_per_s: float = 200.0,
                 n_lo: int = 10_000, n_hi: int = 2_000_000, pool: int = 48) -> list:
    """A Poisson stream (mean ``rate_per_s`` jobs/s) of clustering requests:
    n log-uniform on [10k, 2M], d uniform on {2..8}, blob mixtures as in
    ``batch_256``, and 1-4 follow-up (rho_min, delta_min) re-queries each.

    ``pool`` distinct problems are drawn and every request takes one of them
    at random (with its own arrival time and queries), so that a long trace
    does not need tens of GB of host memory; requests sharing a problem
    share its point array (each request is still clustered from scratch)."""
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(pool):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(rng.integers(2, 9))
        target = float(rng.uniform(20, 200))
        probs.append(_random_problem(rng, f"problem_{i}", n, d, target))
    t = 0.0
    out = []
    for j in range(jobs):
        t += float(rng.exponential(1.0 / rate_per_s))
        src = probs[int(rng.integers(pool))]
        nq = int(rng.integers(1, 5))
        queries = [(max(1, int(src.rho_min * rng.uniform(0.5, 2.0))),
                    max(src.d_cut + 1, int(src.d_cut * rng.uniform(4, 12)))) for _ in range(nq)]
        out.append(Dataset(f"job_{j}", src.points, src.d_cut, src.rho_min, src.delta_min,
                           queries=queries, arrival_s=t, seed=seed))
    return out


def served_problem(seed: int = 6, n: int = 2_000_000, d: int = 8) -> Dataset:
    """One request of the served trace's recipe at a chosen size (the trace
    draws n up to 2M and d up to 8): a blob mixture + 5% noise with its own
    cutoff (mean rho 20-200), rho_min and delta_min."""
    rng = np.random.default_rng(seed)
    target = float(rng.uniform(20, 200))
    ds = _random_problem(rng, f"served_{n}_{d}d", n, d, target)
    ds.seed = seed
    return ds


def random_blobs(seed: int, n: int, d: int, d_cut: int, domain: int = DOMAIN,
                 blobs: int = 4, spread: float = 0.05, dup: int = 0) -> Dataset:
    """Small seeded test problems: a few blobs + uniform noise in
    [0, domain]^d, optionally with ``dup`` exact duplicate points."""
    rng = np.random.default_rng(seed)
    if n == 0:
        return Dataset(f"rand_{seed}", np.zeros((0, d), np.int32), d_cut, 1, d_cut + 1, seed=seed)
    k = max(1, blobs)
    centers = rng.uniform(0, domain, size=(k, d))
    lab = rng.integers(0, k, size=n)
    pts = centers[lab] + rng.standard_normal((n, d)) * spread * domain
    noise = rng.random(n) < 0.1
    pts[noise] = rng.uniform(0, domain, size=(int(noise.sum()), d))
    pts = np.clip(np.rint(pts), 0, domain).astype(np.int32)
    if dup and n > dup:
        pts[n - dup:] = pts[:dup]
    return Dataset(f"rand_{seed}", np.ascontiguousarray(pts), d_cut, 2, 3 * d_cut + 1, seed=seed)


NAMED = {
    "plain_20k_2d": plain_20k_2d,
    "plain_5p8m_3d": plain_5p8m_3d,
    "plain_2m_3d": plain_2m_3d,
    "plain_1m_8d": plain_1m_8d,
    "plain_400k_8d": plain_400k_8d,
    "plain_5p8m_3d_dense": plain_5p8m_3d_dense,
}
