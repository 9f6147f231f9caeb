"""The bench's multi-rank host logic on two gloo ranks (CPU): the barrier, the
slowest-rank time that the whole-job rate divides by, and the reference arm
running on rank 0 only.  Updates shard as independent replicas (no collective
on the data path), so this host logic is all that multi-GPU runs add."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    slowest = bench.max_over_ranks(world, 10.0 + rank)  # rank 1 is the slower one
    rate = bench.aggregate_rate(world, 8192, 5, slowest)
    with open(out % rank, "w") as f:
        json.dump({"slowest": slowest, "rate": rate}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    out = str(tmp_path / "rank%d.json")
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    got = [json.load(open(out % r)) for r in range(2)]
    assert got[0] == got[1]
    assert got[0]["slowest"] == 11.0
    assert got[0]["rate"] == pytest.approx(2 * 8192 * 5 / 0.011)


def test_reference_arm_prints_nothing_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--host-inputs"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
