#!/usr/bin/env python
"""Benchmark of exact Density-Peaks Clustering on GB300.

Metric: exact DPC points/s (rho + delta + labels) on the 5.8M x 3 workload
(50 skewed Gaussian blobs + 2% noise, d_cut calibrated for mean rho ~ 100;
a synthetic stand-in for the paper's Airline set). One step = dpc_density +
dpc_dependent + dpc_label of the whole set through the C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`value` times the steps with the points already in device memory (CUDA
events on the library's stream, L2 flushed between steps); `e2e` times the
same steps from pinned host memory to host results (copies included).
With N > 1 (torchrun) every rank clusters its own replica of the workload
(independent problems: weak scaling, no collective on the data path).
`--impl reference` times the CPU oracle (the plain O(n^2) scan of the
paper's definitions) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact DPC points/s (rho+delta+labels) at 5.8M x 3"
APPROX_METRIC = "Approx-DPC points/s (rho+approximate delta+labels) at 5.8M x 3"


SAPPROX_METRIC = "S-Approx-DPC points/s (rho of picks+approximate delta+labels) at 5.8M x 3"


# the single-dataset workloads' sizes, as the metric names them
SIZE_NAME = {"plain_5p8m_3d": "5.8M x 3", "plain_2m_3d": "2M x 3", "plain_1m_8d": "1M x 8",
             "plain_400k_8d": "400k x 8", "plain_20k_2d": "20k x 2",
             "plain_5p8m_3d_dense": "5.8M x 3, d_cut x 4"}


def metric_for(args) -> str:
    m = {"approx": APPROX_METRIC, "sapprox": SAPPROX_METRIC}.get(args.method, METRIC)
    return m.replace("5.8M x 3", SIZE_NAME.get(args.workload, args.workload))
UNIT = "points/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="plain_5p8m_3d")
    ap.add_argument("--method", choices=["exact", "approx", "sapprox"], default="exact",
                    help="exact DPC, Approx-DPC's dependent points (Section 4.3) or S-Approx-DPC (Section 5)")
    ap.add_argument("--eps", default="0.8", help="S-Approx-DPC's eps (a decimal, or num/den)")
    ap.add_argument("--eps-sweep", default="",
                    help="S-Approx-DPC: comma-separated eps values for a time / Rand-index curve")
    ap.add_argument("--cpu-sample", type=int, default=0, help="oracle sample size (0: automatic)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rate", type=float, default=200.0,
                    help="served_trace: offered jobs/s of the Poisson trace (200 by default)")
    ap.add_argument("--tune", default="",
                    help="tuning knobs for the timed context, key=value[,key=value...] (dpc_set_tuning)")
    return ap.parse_args()


def parse_eps(text: str):
    """S-Approx-DPC's eps as (num, den): "num/den", or a decimal to 10^-6."""
    import math
    if "/" in text:
        a, b = text.split("/")
        return int(a), int(b)
    num, den = int(round(float(text) * 10 ** 6)), 10 ** 6
    g = math.gcd(num, den)
    return num // g, den // g


def parse_tune(text: str) -> dict:
    """Tuning knobs "key=value,key=value" as {key: int}."""
    out = {}
    for item in filter(None, (t.strip() for t in text.split(","))):
        key, sep, val = item.partition("=")
        if not sep or not key.strip():
            raise ValueError(f"--tune expects key=value, got {item!r}")
        out[key.strip()] = int(val)
    return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest of every rank's x (the whole job is as slow as its slowest
    rank); x itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws: int, units_per_rank: float, steps: int, total_ms: float) -> float:
    """Units all ranks processed per second over the slowest rank's time."""
    return ws * units_per_rank * steps / (total_ms / 1e3)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------- oracle leg

def oracle_sample_rate(ds, m: int, seed: int = 7, method: str = "exact", eps=(4, 5)):
    """The oracle, as it stands, on m sampled points of the workload: their
    local density against all n points, then their dependent point (exact:
    a scan of all n points; approx: Approx-DPC's rules, which scan all n
    points for a cell's top; sapprox: S-Approx-DPC's grid of all n points
    and both phases, which scan all n points). Only the time is used. The density order is
    the index order here (the full density array would need the whole
    O(n^2) oracle run); on a uniform sample the exact scan touches the same
    number of higher points on average (half of them)."""
    import numpy as np
    import oracle
    idx = np.random.default_rng(seed).choice(ds.n, size=m, replace=False)
    flat = np.zeros(ds.n, dtype=np.int32)
    t0 = time.perf_counter()
    oracle.rho_subset(ds.points, ds.d_cut, idx)
    if method == "approx":
        oracle.approx_dependent_subset(ds.points, flat, ds.d_cut, idx)
    elif method == "sapprox":
        oracle.sapprox_dependent_subset(ds.points, flat, ds.d_cut, eps[0], eps[1], idx)
    else:
        oracle.dependent_subset(ds.points, flat, idx)
    dt = time.perf_counter() - t0
    return m / dt, dt


def auto_sample(ds) -> int:
    # about 15 s of oracle work on the GPU machine's 16 host cores, which run the
    # sampled oracle at about 8e9 pair tests/s (5.8M x 3: 950 points/s at
    # 1.5 n pair tests per point)
    return min(ds.n, max(200, min(40000, int(1.2e11 / (1.5 * ds.n)))))


# ----------------------------------------------------------------- our arm

def derived_pair_peak(d: int, form: int, sm_mhz) -> dict:
    """Pair-test ceiling from unit counts: 152 SMs x 4 schedulers x 32
    integer lanes at the SM clock seen under load (2070 MHz when none was
    sampled), over the integer operations one pair takes in the kernel's
    form: d + 3 for the expanded form (add, d multiply-adds, shift,
    accumulate), 2d + 2 for the direct 32-bit form, 4d + 3 for 64-bit."""
    mhz = sm_mhz or 2070.0
    ops = d + 3 if form == 2 else (2 * d + 2 if form == 0 else 4 * d + 3)
    lane_ops = 152 * 4 * 32 * mhz * 1e6
    return {"value": lane_ops / ops / 1e9, "unit": "Gpair/s", "ops_per_pair": ops, "sm_mhz": mhz,
            "derivation": f"152 SMs x 4 x 32 lanes x {mhz:.0f} MHz / {ops} integer ops per pair"}


def hbm_peak():
    """(GB/s, source) of the HBM roofline: the measured copy bandwidth, else
    the profiling recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def e2e_roofline(n: int, d: int, info: dict, pair_rate: float, value: float) -> dict:
    """End-to-end points/s roofline: n over the sum of the stages' roofline
    times. Grid, rank sort and labels are HBM-bound, at algorithmic bytes per
    point (kb = key bytes, P = radix passes = key bits / 8 rounded up; one
    histogram pass reads the keys, kb, and each pass reads the keys and the
    values and writes both: 2 kb + 8 bytes): grid = read the input 4d, write key and index kb + 4,
    P passes, gather (index 4, input 4d, record 16 per 4 dims), cells and hash
    8; rank = keys kb + 4, P passes, rank and (rank, index) 20; labels = read
    rho, dep, delta2 (16), write parent and label (8), read parents (4). The
    density and ring passes are ALU-bound: candidate pairs over the measured
    pair rate, each. The open-point searches are data dependent and not
    modelled (zero time), so the bound is optimistic."""
    gbs, src = hbm_peak()
    dp = 1 if d <= 4 else 2

    def sort_bytes(bits):
        kb = 4 if bits <= 32 else 8
        return kb, kb + max(1, (bits + 7) // 8) * (2 * kb + 8)

    kb, gp = sort_bytes(info.get("grid_key_bits") or 32)
    grid_b = n * (4 * d + kb + 4 + gp + 4 + 4 * d + 16 * dp + 8)
    kr, rp = sort_bytes(info.get("rank_key_bits") or 32)
    rank_b = n * (kr + 4 + rp + 20)
    label_b = n * (16 + 8 + 4)
    pairs = info["cand_pairs"]
    ms = {"grid_hbm": grid_b / (gbs * 1e9) * 1e3, "rho_alu": pairs / pair_rate * 1e3,
          "rank_hbm": rank_b / (gbs * 1e9) * 1e3, "ring_alu": pairs / pair_rate * 1e3,
          "open_points": 0.0, "labels_hbm": label_b / (gbs * 1e9) * 1e3}
    total = sum(ms.values())
    bound = n / (total / 1e3)
    return {"stages_ms": ms, "points_per_s": bound, "frac": value / bound, "hbm_gbs": gbs,
            "hbm_source": src, "pair_rate": pair_rate,
            "bytes_per_point": {"grid": grid_b / n, "rank": rank_b / n, "labels": label_b / n}}


def stage_rooflines(n: int, e2e: dict, stages: dict, work: dict, rho_rate: float, ring_rate, ring_src: str) -> dict:
    """Each stage of one step against its own ceiling (the paper's split of
    Ex-DPC's time into rho and delta, Table 6, taken stage by stage): the
    HBM-bound stages at their algorithmic bytes per point (e2e_roofline's
    model) over the stage's CUDA-event time, against the measured copy
    bandwidth; the density and ring passes at candidate pairs over their
    time, against the probe of their own pair test; the open points (tree
    search and brute force, latency bound, no ceiling) as points and tree
    node visits per second."""
    gbs = e2e["hbm_gbs"]
    bpp = e2e["bytes_per_point"]
    pairs = work["cand_pairs"]

    def hbm(key, ms):
        gb = n * bpp[key] / (ms / 1e3) / 1e9 if ms > 0 else 0.0
        return {"bound": "hbm", "ms": ms, "bytes_per_point": bpp[key], "achieved": gb, "peak": gbs,
                "unit": "GB/s", "frac": gb / gbs}

    def alu(ms, peak, src):
        a = pairs / (ms / 1e3) if ms > 0 else 0.0
        return {"bound": "alu", "ms": ms, "pairs": pairs, "achieved": a / 1e9,
                "peak": peak / 1e9 if peak else None, "unit": "Gpair/s", "frac": a / peak if peak else None,
                "peak_source": src}

    rest = stages["ms_rest"]
    return {
        "grid": hbm("grid", stages["ms_grid"]),
        "density": alu(stages["ms_rho"], rho_rate, "dpc_probe_pair_rate, the density kernel's pair form"),
        "rank": hbm("rank", stages["ms_rank"]),
        "ring": alu(stages["ms_ring"], ring_rate, ring_src),
        "open_points": {"bound": "latency", "ms": rest, "points": work["open_after_ring"],
                        "points_per_s": work["open_after_ring"] / (rest / 1e3) if rest > 0 else 0.0,
                        "tree_visits": work["tree_visits"],
                        "visits_per_s": work["tree_visits"] / (rest / 1e3) if rest > 0 else 0.0},
        "labels": hbm("labels", stages["ms_label"]),
    }


GRID_SOURCES = ("grid.cu", "sort.cu", "rho.cu", "delta.cu", "label.cu", "stages.cuh", "dpc_internal.cuh")


def kernel_hbm(workload: str):
    """Achieved DRAM GB/s of the grid, sort, scatter and gather kernels from
    the ncu capture summarized in profiles/ (dram__bytes_read + write over
    gpu__time_duration of each launch, serialized and cold: a lower bound of
    the kernel's rate inside a step), or None when that capture was of
    another workload or another version of the kernels."""
    tpath = os.path.join(ROOT, "profiles", "grid_traffic.json")
    if not os.path.exists(tpath):
        return None
    with open(tpath) as f:
        tj = json.load(f)
    if tj.get("workload") != workload or tj.get("source_sha256") != source_digest(GRID_SOURCES):
        return None
    gbs, _ = hbm_peak()
    out = {}
    for k, e in tj["kernels"].items():
        rate = e["dram_bytes"] / (e["ns"] * 1e-9) / 1e9
        out[k] = {"dram_bytes": e["dram_bytes"], "us": e["ns"] / 1e3, "achieved": rate, "unit": "GB/s",
                  "frac": rate / gbs}
    return {"kernels": out, "peak": gbs, "summary": tj.get("summary")}


RHO_SOURCES = ("rho.cu", "stages.cuh", "dpc_internal.cuh")


def source_digest(names) -> str:
    """sha256 over the named kernel sources (csrc/)."""
    import hashlib
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2207_04649_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def rho_source_digest() -> str:
    """sha256 over the density kernels' sources: DRAM counters taken on
    another version of them do not describe this build."""
    import hashlib
    h = hashlib.sha256()
    for f in RHO_SOURCES:
        with open(os.path.join(ROOT, "paper_2207_04649_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def rho_traffic(workload: str, key: str = "dram_bytes_per_launch"):
    """DRAM bytes (read + write) of one step's density pair launches (key
    dram_bytes_per_launch: dense + sparse kernels; *_dense: the dense kernel),
    from the ncu capture summarized in profiles/, or None when that capture
    was of another workload or another version of the kernels."""
    tpath = os.path.join(ROOT, "profiles", "rho_traffic.json")
    if not os.path.exists(tpath):
        return None
    with open(tpath) as f:
        tj = json.load(f)
    if tj.get("workload") != workload or tj.get("source_sha256") != rho_source_digest():
        return None
    return tj.get(key)


def run_ours(args):
    import numpy as np
    import torch
    import workloads
    import paper_2207_04649_gb300 as dpc

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    ds = workloads.NAMED[args.workload]()
    n, d = ds.n, ds.d
    dev = torch.device("cuda", local)
    pts = torch.from_numpy(ds.points).to(dev)
    rho = torch.empty(n, dtype=torch.int32, device=dev)
    dep = torch.empty(n, dtype=torch.int32, device=dev)
    d2 = torch.empty(n, dtype=torch.int64, device=dev)
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2 (126 MB)
    ctx = dpc.Context(device=local, profiling=True)
    knobs = parse_tune(args.tune)
    if knobs:
        ctx.tune(**knobs)
    st = ctx.stream

    approx = args.method == "approx"
    sapprox = args.method == "sapprox"
    eps = parse_eps(args.eps)
    pick = torch.empty(n, dtype=torch.uint8, device=dev)

    def step():
        if sapprox:
            h = ctx.sapprox(pts, ds.d_cut, eps, rho, dep, d2, pick)
        else:
            h = ctx.density(pts, ds.d_cut, rho)
            if approx:
                h.dependent_approx(dep, d2)
            else:
                h.dependent(dep, d2)
        nc = h.label(ds.rho_min, ds.delta_min, lab)
        info = h.info()
        h.release()
        return nc, info

    torch.cuda.synchronize()
    winfo = None
    for _ in range(args.warmup):
        _, winfo = step()
    torch.cuda.synchronize()
    # integer-ALU ceiling of the pair test in the form the kernel runs (before
    # anything is timed)
    pair_mode = winfo["pair_mode"] if winfo else 0
    probe_rate, _ = dpc.dpc_probe_pair_rate(local, d, pair_mode)
    if pair_mode == 2:
        ring_rate, _ = dpc.dpc_probe_pair_rate(local, d, 3)
        ring_src = "measured: the ring search's pair test (expanded form, rank compare, least packed key) " \
                   "with operands in registers on all SMs (dpc_probe_pair_rate mode 3), same run"
    else:
        ring_rate = probe_rate
        ring_src = f"measured: the density pair test (form {pair_mode}) only, a ceiling above the ring's"

    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = dpc.dpc_kernel_launches()
    evs = []
    infos = []
    for _ in range(args.steps):
        with torch.cuda.stream(st):
            flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        nc, info = step()
        b.record(st)
        evs.append((a, b))
        infos.append(info)
    torch.cuda.synchronize()
    launches = dpc.dpc_kernel_launches() - l0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    value = whole_job_rate(ws, n, args.steps, total_ms)

    # end to end: pinned host input -> host results, through the same ABI
    h_pts = torch.from_numpy(ds.points).pin_memory().numpy()
    h_rho = torch.empty(n, dtype=torch.int32).pin_memory().numpy()
    h_dep = torch.empty(n, dtype=torch.int32).pin_memory().numpy()
    h_d2 = torch.empty(n, dtype=torch.int64).pin_memory().numpy()
    h_lab = torch.empty(n, dtype=torch.int32).pin_memory().numpy()
    h_pick = torch.empty(n, dtype=torch.uint8).pin_memory().numpy()
    e2e_s = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if sapprox or approx:
            if sapprox:
                h = ctx.sapprox(h_pts, ds.d_cut, eps, h_rho, h_dep, h_d2, h_pick)
            else:
                h = ctx.density(h_pts, ds.d_cut, h_rho)
                h.dependent_approx(h_dep, h_d2)
            h.label(ds.rho_min, ds.delta_min, h_lab)
            h.release()
        else:
            # the one-call entry point: results leave the device while later stages run
            ctx.cluster(h_pts, ds.d_cut, ds.rho_min, ds.delta_min, h_rho, h_dep, h_d2, h_lab)
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_s.append(t1 - t0)
    e2e_total = max_over_ranks(sum(e2e_s), dist, dev)
    e2e_value = whole_job_rate(ws, n, len(e2e_s), 1e3 * e2e_total)

    # roofline of the dominant density kernel (dense cells; ALU bound), and of
    # the density stage as a whole (dense + sparse cells)
    rho_ms = statistics.mean(i["ms_rho"] for i in infos)
    dense_ms = statistics.mean(i["ms_rho_dense"] for i in infos)
    pairs = infos[-1]["cand_pairs"]
    dpairs = infos[-1]["dense_pairs"]
    achieved = pairs / (rho_ms / 1e3) if rho_ms > 0 else 0.0
    dachieved = dpairs / (dense_ms / 1e3) if dense_ms > 0 else 0.0
    # the DRAM capture covers the density kernels over every point, with the
    # default knobs, only
    all_points = infos[-1].get("density_path", 0) == 0
    traffic = rho_traffic(args.workload) if all_points and not knobs else None
    dtraffic = rho_traffic(args.workload, "dram_bytes_per_launch_dense") if all_points and not knobs else None

    if dpairs > 0:
        queries = "each grid cell's picks" if infos[-1].get("density_path") == 3 else "dense cells"
        kname = "k_rho_dense_bulk" if knobs.get("rho_bulk") and all_points and d <= 4 and pair_mode != 1 else "k_rho_dense"
        roofline = {"bound": "alu", "kernel": f"{kname} ({queries}, pair form {pair_mode})",
                    "achieved": dachieved / 1e9, "peak": probe_rate / 1e9, "unit": "Gpair/s",
                    "frac": dachieved / probe_rate, "traffic": dtraffic,
                    "pairs_per_launch": dpairs, "ms_per_launch": dense_ms,
                    "density_stage": {"kernels": "k_rho_dense + k_rho_sparse" if all_points else
                                      "pick lists, pick items, k_rho_dense", "achieved": achieved / 1e9,
                                      "frac": achieved / probe_rate, "traffic": traffic,
                                      "pairs_per_step": pairs, "ms_per_step": rho_ms},
                    "peak_source": "measured: the kernel's own pair test (form "
                                   f"{pair_mode}, {'64' if pair_mode == 1 else '32'}-bit) with operands "
                                   "in registers on all SMs (dpc_probe_pair_rate), same run",
                    "pair_mode": pair_mode,
                    "peak_derived": derived_pair_peak(d, pair_mode, clk.get("sm_mhz"))}
    else:
        # S-Approx-DPC's pick path with few candidates per pick: its density
        # kernel (one warp per pick, or per grid cell) runs the direct 64-bit
        # pair test
        p64, _ = dpc.dpc_probe_pair_rate(local, d, 1)
        kname = ("k_sap_rho_cells (one warp per grid cell" if infos[-1].get("density_path") == 2
                 else "k_sap_rho (one warp per pick")
        roofline = {"bound": "alu", "kernel": f"{kname}, direct 64-bit pair test)",
                    "achieved": achieved / 1e9, "peak": p64 / 1e9, "unit": "Gpair/s",
                    "frac": achieved / p64, "traffic": None, "pairs_per_launch": pairs, "ms_per_launch": rho_ms,
                    "peak_source": "measured: the direct 64-bit pair test with operands in registers on all "
                                   "SMs (dpc_probe_pair_rate mode 1), same run",
                    "pair_mode": 1, "peak_derived": derived_pair_peak(d, 1, clk.get("sm_mhz"))}

    accuracy = None
    if approx or sapprox:
        # Rand index of the Approx-DPC labels against the exact labels of the
        # same set (the paper's accuracy measure, Section 5), and the center
        # guarantee of Section 4.4
        from paper_2207_04649_gb300 import evaluate
        h = ctx.density(pts, ds.d_cut)
        elab = torch.empty_like(lab)
        h.dependent()
        h.label(ds.rho_min, ds.delta_min, elab)
        h.release()
        torch.cuda.synchronize()
        a_np, e_np = lab.cpu().numpy(), elab.cpu().numpy()
        idx = np.arange(n)
        accuracy = {"rand_index_vs_exact": evaluate.rand_index(a_np, e_np),
                    "same_centers": bool(np.array_equal(a_np == idx, e_np == idx))}
        if approx:
            accuracy["tops_to_exact_search"] = int(infos[-1]["open_after_ring"])
        else:
            accuracy.update({"eps": list(eps), "picks": int(infos[-1]["picks"]),
                             "second_phase": int(infos[-1]["second_phase"]),
                             "to_tree_or_brute_force": int(infos[-1]["open_after_ring"])})

    eps_curve = None
    if sapprox and args.eps_sweep:
        eps_curve = sapprox_eps_curve(ctx, pts, ds, [parse_eps(t) for t in args.eps_sweep.split(",")],
                                      lab, elab, flush)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        m = args.cpu_sample or auto_sample(ds)
        rate, dt = oracle_sample_rate(ds, m, method=args.method, eps=eps)
        cpu = {"value": rate, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
               "sample": f"{m} random points of the {n}-point set: rho against all n points and the "
                         f"{args.method} dependent-point step over all n points ({dt:.1f} s)",
               "full_run_s_extrapolated": n / rate}

    if dist:
        dist.barrier()
    e2e = e2e_roofline(n, d, infos[-1], probe_rate, value)
    stages = {k: statistics.mean(i[k] for i in infos)
              for k in ("ms_grid", "ms_rho", "ms_rank", "ms_ring", "ms_rest", "ms_label")}
    work = {k: infos[-1][k] for k in ("cells", "dense_cells", "work_items", "cand_pairs", "dense_pairs",
                                      "open_after_ring", "brute_points", "grid_dims", "pair_bits",
                                      "tree_visits", "tree_pairs")}
    if rank == 0:
        line = {
            "metric": metric_for(args), "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded Gaussian-blob mixture, int32 coordinates)",
            "config": {"workload": args.workload, "method": args.method,
                       **({"eps": f"{eps[0]}/{eps[1]}"} if sapprox else {}),
                       "n": n, "d": d, "d_cut": ds.d_cut, "rho_min": ds.rho_min,
                       "delta_min": ds.delta_min, "parallelism": f"replicas x{ws}",
                       "l2": "flushed between steps (256 MB write)",
                       "mean_rho": float(rho.double().mean().item()), "n_centers": int(nc),
                       **({"tune": knobs} if knobs else {})},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * d * 4,
                    "d2h_bytes_per_step": n * (4 + 4 + 8 + 4 + (1 if sapprox else 0)) + 8},
            "roofline": roofline,
            "e2e_roofline": e2e,
            "stages_ms": stages,
            "stage_rooflines": stage_rooflines(n, e2e, stages, work, probe_rate, ring_rate, ring_src),
            "kernel_hbm": kernel_hbm(args.workload) if not knobs else None,
            "work": work,
            "cpu_baseline": cpu,
            "clocks": clk,
            "gpu_launches": launches,
        }
        if accuracy is not None:
            line["accuracy"] = accuracy
        if eps_curve is not None:
            line["eps_curve"] = eps_curve
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def sapprox_eps_curve(ctx, pts, ds, eps_list, lab, elab, flush, reps: int = 3):
    """Time (device-resident, L2 flushed, mean of reps after one warm-up) and
    Rand index against the exact labels of S-Approx-DPC for every eps (the
    paper's Table 5 on this workload), plus the exact path's own time."""
    import torch
    from paper_2207_04649_gb300 import evaluate
    st = ctx.stream
    e_np = elab.cpu().numpy()

    def timed(run):
        run()
        ms = []
        for _ in range(reps):
            with torch.cuda.stream(st):
                flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            out = run()
            b.record(st)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.mean(ms), out

    def exact():
        h = ctx.density(pts, ds.d_cut)
        nc = h.label(ds.rho_min, ds.delta_min)
        h.release()
        return nc

    ex_ms, ex_nc = timed(exact)
    curve = [{"eps": "exact", "ms": ex_ms, "n_centers": ex_nc, "rand_index": 1.0}]
    for eps in eps_list:
        def run():
            h = ctx.sapprox(pts, ds.d_cut, eps)
            nc = h.label(ds.rho_min, ds.delta_min, lab)
            info = h.info()
            h.release()
            return nc, info
        ms, (nc, info) = timed(run)
        a_np = lab.cpu().numpy()
        curve.append({"eps": f"{eps[0]}/{eps[1]}", "ms": ms, "n_centers": nc, "picks": int(info["picks"]),
                      "second_phase": int(info["second_phase"]),
                      "rand_index": evaluate.rand_index(a_np, e_np)})
    return curve


# ----------------------------------------------------------- reference arm

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import workloads
    ds = workloads.NAMED[args.workload]()
    m = args.cpu_sample or max(100, auto_sample(ds) // 4)
    eps = parse_eps(args.eps)
    for _ in range(args.warmup):
        oracle_sample_rate(ds, max(20, m // 10), method=args.method, eps=eps)
    times = []
    for i in range(args.steps):
        _, dt = oracle_sample_rate(ds, m, seed=100 + i, method=args.method, eps=eps)
        times.append(dt)
    total = sum(times)
    value = m * len(times) / total
    sample = (f"{m} random points per step of the {ds.n}-point set: rho against all n points and the "
              f"dependent-point scan over all n points")
    line = {
        "impl": "reference", "metric": metric_for(args), "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": args.workload, "method": args.method, "n": ds.n, "d": ds.d, "d_cut": ds.d_cut},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------- batched and served forms

BATCH_METRIC = "batched exact DPC jobs/s (256 datasets, n 1k-200k, d 2-4)"
SERVED_METRIC = "served exact DPC jobs/s (Poisson {rate:g} jobs/s, n 10k-2M, d 2-8, 1-4 re-queries)"


def run_batched(args):
    """Workload batch_256: one step = the 256 datasets clustered as one batch
    (dpc_submit x 256 + dpc_flush: every stage one launch over all of them),
    against the same datasets one at a time (submit + flush per dataset)."""
    import numpy as np
    import torch
    import workloads
    import paper_2207_04649_gb300 as dpc

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    probs = workloads.batch_256()
    dev = torch.device("cuda", local)
    n_tot = sum(p.n for p in probs)
    ctx = dpc.Context(device=local, mode=0, profiling=True)
    knobs = parse_tune(args.tune)
    if knobs:
        ctx.tune(**knobs)
    st = ctx.stream
    djobs = [dpc.Job(torch.from_numpy(p.points).to(dev), p.d_cut, [(p.rho_min, p.delta_min)]) for p in probs]
    hjobs = [dpc.Job(torch.from_numpy(p.points).pin_memory().numpy(), p.d_cut, [(p.rho_min, p.delta_min)],
                     pinned=True)
             for p in probs]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    def run(jobs, together=True):
        if together:
            for j in jobs:
                ctx.submit(j)
            ctx.flush()
        else:
            for j in jobs:
                ctx.submit(j)
                ctx.flush()
        for j in jobs:
            s, _ = ctx.poll(j.ticket)
            if s != dpc.DPC_OK:
                raise RuntimeError(f"job failed with status {s}")

    def timed(jobs, steps, together=True, events=True):
        ms = []
        for _ in range(steps):
            with torch.cuda.stream(st):
                flush.fill_(1)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            a.record(st)
            run(jobs, together)
            b.record(st)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b) if events else 1e3 * (time.perf_counter() - t0))
        return ms

    for _ in range(args.warmup):
        run(djobs)
    # knobs from the project's autotuner, run on this batch before timing
    tuned = ctx.autotune(djobs, repeats=2)
    run(djobs)
    # a batch mixes d = 2, 3 and 4: the ceiling quoted is the d = 3 pair test
    # in the expanded 32-bit form (between the d = 2 and d = 4 rates)
    probe_rate = dpc.dpc_probe_pair_rate(local, 3, 2)[0]
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    l0 = dpc.dpc_kernel_launches()
    ms = timed(djobs, args.steps)
    launches = dpc.dpc_kernel_launches() - l0
    clk = clocks.stop()
    info = ctx.last_batch_info()
    total_ms = max_over_ranks(sum(ms), dist, dev)
    value = whole_job_rate(ws, len(probs), args.steps, total_ms)
    # the same datasets one at a time (device inputs), and host-buffer runs
    run(djobs, together=False)
    alone_ms = sum(timed(djobs, 1, together=False))
    run(hjobs)
    e2e_ms = max_over_ranks(sum(timed(hjobs, args.steps, events=False)), dist, dev)
    e2e_value = whole_job_rate(ws, len(probs), args.steps, e2e_ms)
    achieved = info["cand_pairs"] / (info["ms_rho"] / 1e3) if info["ms_rho"] > 0 else 0.0
    if rank == 0:
        line = {
            "metric": BATCH_METRIC, "value": value, "unit": "jobs/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded Gaussian-blob mixtures + 5% noise, int32 coordinates)",
            "config": {"workload": "batch_256", "jobs": len(probs), "points": n_tot,
                       "parallelism": f"replicas x{ws}", "l2": "flushed between steps (256 MB write)",
                       "points_per_s": value * n_tot / len(probs), "autotuned": tuned,
                       **({"tune": knobs} if knobs else {}),
                       "one_at_a_time_jobs_per_s": len(probs) / (alone_ms / 1e3),
                       "batched_over_one_at_a_time": (len(probs) / (total_ms / args.steps / 1e3))
                       / (len(probs) / (alone_ms / 1e3))},
            "e2e": {"value": e2e_value, "unit": "jobs/s", "h2d_bytes_per_step": sum(p.n * p.d * 4 for p in probs),
                    "d2h_bytes_per_step": sum(p.n * 20 + 8 for p in probs)},
            "roofline": {"bound": "alu", "kernel": "density pair kernels (dense + sparse cells), whole batch",
                         "achieved": achieved / 1e9, "peak": probe_rate / 1e9, "unit": "Gpair/s",
                         "frac": achieved / probe_rate, "traffic": None,
                         "peak_source": "measured: dpc_probe_pair_rate(d=3, expanded 32-bit form), same "
                                        "run; the batch mixes d = 2, 3, 4",
                         "pairs_per_launch": info["cand_pairs"], "ms_per_launch": info["ms_rho"]},
            "stages_ms": {k: info[k] for k in ("ms_grid", "ms_rho", "ms_rank", "ms_ring", "ms_rest")},
            "work": {k: info[k] for k in ("n", "cells", "cand_pairs", "open_after_ring", "brute_points",
                                          "tree_visits")},
            "cpu_baseline": None,
            "clocks": clk,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def _replay(dpc, ctx, trace, t0):
    """Submit the trace's jobs at their arrival times (host buffers) from one
    thread while another collects them in order; per-job latency is
    submit -> results in host memory."""
    import threading
    jobs = [None] * len(trace)
    ready = [threading.Event() for _ in trace]

    def submitter():
        for i, ds in enumerate(trace):
            delay = t0 + ds.arrival_s - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            j = dpc.Job(ds.points, ds.d_cut, ds.queries)
            ctx.submit(j)
            jobs[i] = j
            ready[i].set()

    th = threading.Thread(target=submitter)
    th.start()
    lat = []
    done_at = []
    for i in range(len(trace)):
        ready[i].wait()
        s, r = ctx.wait(jobs[i].ticket)
        if s != dpc.DPC_OK:
            raise RuntimeError(f"job {i} failed with status {s}")
        lat.append(r.queue_ms + r.run_ms)
        done_at.append(time.perf_counter())
        jobs[i] = None
    th.join()
    return lat, done_at


def run_served(args):
    """Workload served_trace: the Poisson trace replayed in real time against
    the served mode (continuous batching under a 150 GB cap), and the same
    trace against one-job-at-a-time service."""
    import numpy as np
    import torch
    import workloads
    import paper_2207_04649_gb300 as dpc

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    trace = workloads.served_trace(rate_per_s=args.rate)
    warm = workloads.served_trace(seed=6, jobs=max(8, args.warmup * 8), pool=8)

    def serve(max_batch):
        ctx = dpc.Context(device=local, mode=1, hbm_cap_bytes=150 << 30, max_inflight=2)
        ctx.tune(max_batch_jobs=max_batch)
        _replay(dpc, ctx, warm, time.perf_counter())
        l0 = dpc.dpc_kernel_launches()
        t0 = time.perf_counter()
        lat, done_at = _replay(dpc, ctx, trace, t0)
        launches = dpc.dpc_kernel_launches() - l0
        span = max(done_at) - t0
        ctx.close()
        return lat, span, launches

    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    lat, span, launches = serve(64)
    clk = clocks.stop()
    span = max_over_ranks(span, dist, dev)
    lat1, span1, _ = serve(1)
    span1 = max_over_ranks(span1, dist, dev)
    pts = sum(ds.n for ds in trace)
    q = lambda a, f: float(np.percentile(np.asarray(a), f))
    value = whole_job_rate(ws, len(trace), 1, 1e3 * span)
    if rank == 0:
        line = {
            "metric": SERVED_METRIC.format(rate=args.rate), "value": value, "unit": "jobs/s", "n_gpus": ws,
            "steps": 1,
            "warmup": len(warm), "ms_per_step": 1e3 * span, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded Poisson trace of Gaussian-blob mixtures, int32 coordinates)",
            "config": {"workload": "served_trace", "jobs": len(trace), "offered_jobs_per_s": args.rate,
                       "trace_s": trace[-1].arrival_s, "points": pts, "hbm_cap_gb": 150,
                       "parallelism": f"replicas x{ws}",
                       "l2": "inputs are copied from host memory for every job",
                       "p50_ms": q(lat, 50), "p99_ms": q(lat, 99),
                       "one_at_a_time": {"jobs_per_s": whole_job_rate(ws, len(trace), 1, 1e3 * span1),
                                         "p50_ms": q(lat1, 50),
                                         "p99_ms": q(lat1, 99)}},
            "e2e": {"value": value, "unit": "jobs/s", "h2d_bytes_per_step": sum(ds.n * ds.d * 4 for ds in trace),
                    "d2h_bytes_per_step": sum(ds.n * (16 + 4 * len(ds.queries)) + 8 * len(ds.queries)
                                              for ds in trace)},
            "roofline": None,
            "cpu_baseline": None,
            "clocks": clk,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch_256":
        run_batched(args)
    elif args.workload == "served_trace":
        run_served(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
