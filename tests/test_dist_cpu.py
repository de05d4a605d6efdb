"""Multi-rank host logic of the bench on the CPU (gloo): the run is replicas, one
independent box per rank, so the only exchange is the max-over-ranks of the timings."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    got_ws, got_rank, _ = bench.dist_env()
    t = bench.max_over_ranks(1.0 + 1.5 * rank, dist, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, f"r{rank}.json"), "w") as f:
        json.dump(dict(ws=got_ws, rank=got_rank, t=t), f)


@pytest.mark.parametrize("ws", [2, 3])
def test_max_over_ranks_gloo(tmp_path, ws):
    mp.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    for r in range(ws):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d["ws"] == ws and d["rank"] == r
        assert d["t"] == 1.0 + 1.5 * (ws - 1)   # the slowest rank's time, on every rank
    assert bench.max_over_ranks(3.25, None, None) == 3.25


def _bench(args, rank, ws):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_runs_on_rank0_only():
    args = ["--impl", "reference", "--n", "32", "--steps", "2", "--warmup", "1", "--gpus", "2"]
    r1 = _bench(args, 1, 2)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = _bench(args, 0, 2)
    assert r0.returncode == 0, r0.stderr
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    for k in ("metric", "unit", "ms_per_step", "cpu_baseline", "e2e", "config"):
        assert k in line


def test_profiled_traffic_reads_summary_and_checks_source(tmp_path, monkeypatch):
    """The roofline's traffic comes from the committed ncu summary only while its recorded
    source hash equals the current kernel sources' (a note after the hash is allowed)."""
    p = tmp_path / "fwd.txt"
    monkeypatch.setattr(bench, "PROFILE_F32", str(p))
    h = bench.kernel_source_hash()
    p.write_text(f"# header: x\nkernel_source_sha: {h}  (files)\ndram_bytes_per_launch: 123\n")
    assert bench.profiled_traffic() == 123.0
    p.write_text("kernel_source_sha: 0000000000000000\ndram_bytes_per_launch: 123\n")
    assert bench.profiled_traffic() is None
    p.write_text("kernel_source_sha:\ndram_bytes_per_launch: 123\n")
    assert bench.profiled_traffic() is None
