"""The multi-process host logic of bench.py, on CPU with gloo and two ranks:
the time per step reported for N replicas is the slowest replica's (max over
ranks), and the reference arm runs and prints on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, values, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        out[rank] = bench.max_over_ranks(values[rank], world, "cpu")
    finally:
        dist.destroy_process_group()


def test_time_per_step_is_the_max_over_ranks():
    import torch.multiprocessing as mp
    values = [12.5, 40.25]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, _free_port(), values, out), nprocs=2, join=True)
        assert dict(out) == {0: 40.25, 1: 40.25}


def test_single_process_keeps_its_own_time():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1"], env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
