"""The N > 1 host path of bench.py on CPU: world-size-2 gloo process groups and
torchrun launches, no GPU.

On N GPUs the workload runs as N independent replicas (the path does not
exchange data between ranks): the job's time is the slowest rank's, taken
with an all-reduce MAX after a barrier, and the whole-job value counts every
rank's units. The reference arm runs on rank 0 alone; the other ranks exit 0
without output.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier_if_group()
    local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    slowest = bench.max_over_ranks(local_ms, "cpu")
    rate = bench.whole_job_rate(100.0, 3, world, slowest)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "rate": rate}, f)


def test_max_over_ranks_and_whole_job_rate_with_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    port = _free_port()
    torch.multiprocessing.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                                          start_method="spawn")
    for r in range(2):
        got = json.load(open(tmp_path / f"rank{r}.json"))
        assert got["slowest"] == 15.0  # every rank sees the slowest rank's time
        assert got["rate"] == pytest.approx(2 * 3 * 100.0 / 0.015)


def test_single_rank_helpers_need_no_process_group():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    bench.barrier_if_group()
    assert bench.max_over_ranks(7.5, "cpu") == 7.5
    assert bench.whole_job_rate(10.0, 2, 1, 4.0) == pytest.approx(5000.0)


def _json_lines(text):
    return [json.loads(line) for line in text.splitlines() if line.startswith("{")]


def test_reference_arm_prints_one_line():
    pytest.importorskip("torch")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "300", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_under_torchrun_two_ranks():
    """The torchrun launch form for N = 2: rank 0 alone prints the line."""
    pytest.importorskip("torch")
    port = _free_port()
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
                        "--gpus", "2", "--num-nodes", "300", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2
