"""The N > 1 bench path on the CPU: world_size-2 gloo process groups for the
rank reduction, and the reference arm under torchrun (rank 0 alone prints
one line; the other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    # every rank timed its own replica; the job is as slow as the slowest
    own_ms = 100.0 + 50.0 * rank
    total = bench.max_over_ranks(own_ms, dist, "cpu")
    value = bench.whole_job_rate(ws, 1000, 4, total)
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"total": total, "value": value}, f)
    dist.destroy_process_group()


def test_max_over_ranks_with_gloo(tmp_path):
    import torch.multiprocessing as mp
    ws = 2
    port = free_port()
    mp.start_processes(_rank_main, args=(ws, port, str(tmp_path)), nprocs=ws, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    for r in res:
        assert r["total"] == 150.0
        # 2 ranks x 1000 units x 4 steps in 150 ms
        assert r["value"] == pytest.approx(2 * 1000 * 4 / 0.150)


def test_single_process_helpers():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(1, 5_800_000, 10, 111.5) == pytest.approx(5_800_000 * 10 / 0.1115)
    p = bench.derived_pair_peak(3, 2, 2070.0)
    assert p["ops_per_pair"] == 6 and p["value"] == pytest.approx(152 * 128 * 2.07e9 / 6 / 1e9)


def test_reference_arm_under_torchrun():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--workload", "plain_20k_2d", "--steps", "2",
           "--warmup", "1", "--cpu-sample", "40"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0


@pytest.mark.parametrize("method", ["approx", "sapprox"])
def test_reference_arm_approximate_methods(method):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "plain_20k_2d",
           "--method", method, "--eps", "3/5", "--steps", "1", "--warmup", "1", "--cpu-sample", "30"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    line = json.loads(lines[-1])
    assert line["impl"] == "reference" and line["config"]["method"] == method and line["value"] > 0
    assert line["metric"].startswith("S-Approx-DPC" if method == "sapprox" else "Approx-DPC")


def test_parse_tune():
    import bench
    assert bench.parse_tune("") == {}
    assert bench.parse_tune("rho_bulk=1") == {"rho_bulk": 1}
    assert bench.parse_tune(" kch=64, sapprox_path=2 ,") == {"kch": 64, "sapprox_path": 2}
    with pytest.raises(ValueError):
        bench.parse_tune("kch")
    with pytest.raises(ValueError):
        bench.parse_tune("kch=x")


def test_parse_eps():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.parse_eps("0.8") == (4, 5)
    assert bench.parse_eps("3/7") == (3, 7)
    assert bench.parse_eps("1") == (1, 1)


def test_e2e_roofline_model():
    sys.path.insert(0, ROOT)
    import bench
    info = {"grid_key_bits": 30, "rank_key_bits": 23, "cand_pairs": 3_694_000_000}
    r = bench.e2e_roofline(5_800_000, 3, info, 5.1e12, 5.27e8)
    # 3-d: a histogram read of the 32-bit keys (4 B), then 4 grid passes
    # (key and value read and written, 16 B each); 3 rank passes
    assert r["bytes_per_point"]["grid"] == 12 + 8 + 4 + 64 + 4 + 12 + 16 + 8
    assert r["bytes_per_point"]["rank"] == 8 + 4 + 48 + 20
    assert abs(r["stages_ms"]["rho_alu"] - 3.694e9 / 5.1e12 * 1e3) < 1e-9
    assert r["stages_ms"]["open_points"] == 0.0
    assert abs(r["points_per_s"] - 5_800_000 / (sum(r["stages_ms"].values()) / 1e3)) < 1e-3
    assert 0 < r["frac"] < 1


def test_stage_rooflines_model():
    sys.path.insert(0, ROOT)
    import bench
    info = {"grid_key_bits": 30, "rank_key_bits": 23, "cand_pairs": 3_694_000_000}
    e2e = bench.e2e_roofline(5_800_000, 3, info, 5.1e12, 5.27e8)
    stages = {"ms_grid": 1.5, "ms_rho": 1.85, "ms_rank": 0.3, "ms_ring": 2.6, "ms_rest": 2.4, "ms_label": 0.2}
    work = {"cand_pairs": 3_694_000_000, "open_after_ring": 986_000, "tree_visits": 60_000_000}
    r = bench.stage_rooflines(5_800_000, e2e, stages, work, 5.1e12, 4.0e12, "probe")
    g = r["grid"]
    assert g["bound"] == "hbm" and abs(g["achieved"] - 5_800_000 * g["bytes_per_point"] / 1.5e-3 / 1e9) < 1e-6
    assert abs(g["frac"] - g["achieved"] / e2e["hbm_gbs"]) < 1e-12
    assert abs(r["density"]["achieved"] - 3.694e9 / 1.85e-3 / 1e9) < 1e-6
    assert abs(r["ring"]["frac"] - 3.694e9 / 2.6e-3 / 4.0e12) < 1e-12
    assert abs(r["open_points"]["visits_per_s"] - 6e7 / 2.4e-3) < 1e-3
    assert r["labels"]["bytes_per_point"] == 28
