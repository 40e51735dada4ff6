"""The multi-rank host logic of bench.py on CPU ranks (gloo, world size 2).

Frames are independent, so N GPUs run N replicas with no exchange on the data
path; the only collective is the host-side reduction of the timing (max over
ranks) and of the pair counts (sum), which these tests run on gloo."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as td

    sys.path.insert(0, ROOT)
    import bench

    td.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r evaluated (r + 1) * 1e9 pairs in (1 + r) seconds
        value, t_max = bench.aggregate_throughput(td, (rank + 1) * 1e9, 1.0 + rank)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"value": value, "t_max": t_max}, f)
    finally:
        td.destroy_process_group()


def test_aggregate_throughput_over_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    port = free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        got = json.load(open(tmp_path / f"rank{r}.json"))
        assert got["t_max"] == pytest.approx(2.0)
        assert got["value"] == pytest.approx(3e9 / 2.0 / 1e9)  # (1 + 2) Gpairs over the slowest 2 s


def test_single_rank_aggregate_is_local():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate_throughput(None, 5e9, 2.0) == (pytest.approx(2.5), 2.0)


def test_reference_arm_prints_once_under_two_ranks():
    """`bench.py --impl reference` under torchrun: rank 0 times the oracle and
    prints the one JSON line, rank 1 exits 0 without work."""
    pytest.importorskip("torch")
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--particles", "3000", "--nbins", "1000", "--steps", "1",
           "--warmup", "3", "--ref-seconds", "0.3"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
