"""The multi-GPU path of bench.py is replicas only: N independent problems,
one per rank, timed as the slowest rank.  These CPU tests run that host
logic with two gloo ranks (no GPU) and check the reference arm's ranks."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = 100.0 + 50.0 * rank          # rank 1 is the slow one
    value, tot = bench.replica_value(local, 1000, 2, dist, torch.device("cpu"))
    out[rank] = (value, tot)
    dist.destroy_process_group()


def test_replica_value_takes_the_slowest_rank():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        value, tot = res[rank]
        assert tot == 150.0
        assert abs(value - 2 * 1000 * 2 / 0.150) < 1e-6


def test_replica_value_single_process():
    value, tot = bench.replica_value(200.0, 500, 4)
    assert tot == 200.0 and abs(value - 500 * 4 / 0.2) < 1e-9


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
