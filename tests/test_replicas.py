"""Replica (data-parallel over views) aggregation of bench.py on 2 gloo ranks (CPU).

Views are independent, so the multi-GPU path is replicas with no data-path collective:
each rank renders its own poses; the job's throughput is all ranks' frames over the slowest
rank's time.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 if rank == 0 else 250.0          # rank 1 is the slow one
    fps, tot = bench.aggregate(ms, 8, dist, "cpu")
    poses = [bench.replica_pose(i, rank) for i in range(4)]
    q.put((rank, fps, tot, poses))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, fps0, tot0, poses0), (_, fps1, tot1, poses1) = res
    assert tot0 == tot1 == 250.0
    assert fps0 == fps1 == pytest.approx(2 * 8 / 0.25)
    assert poses0 != poses1                     # ranks render different poses


def test_bench_gpus_2_spawns_two_ranks_that_agree():
    """`bench.py --gpus 2` run without a launcher starts two ranks itself (torchrun on
    127.0.0.1); here with gloo ranks on the CPU: rank r reports 10 * (r + 1) ms for 8 frames
    and rank 0 prints the job's aggregate over both ranks."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--replica-selftest"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1                       # rank 0 alone prints
    rec = lines[0]
    assert rec["world"] == 2 and rec["slowest_ms"] == 20.0
    assert rec["value"] == pytest.approx(2 * 8 / 0.020)
