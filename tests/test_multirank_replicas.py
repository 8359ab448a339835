"""Multi-GPU runs are replicas: every rank solves its own instances and the
only exchange is the benchmark's timing reduction (the job lasts as long as
its slowest rank).  That reduction and the whole-job rate are checked here
with two gloo ranks on the CPU."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, outdir):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 1 + r seconds for 3 solves
        value, max_s = bench.job_throughput(1.0 + rank, 3, dist, "cpu")
        with open(os.path.join(outdir, f"r{rank}.json"), "w") as f:
            json.dump({"value": value, "max_s": max_s}, f)
    finally:
        dist.destroy_process_group()


def test_replica_throughput_uses_slowest_rank(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    for r in range(world):
        got = json.load(open(tmp_path / f"r{r}.json"))
        assert got["max_s"] == 2.0
        assert got["value"] == pytest.approx(world * 3 / 2.0)


def test_single_process_throughput():
    import bench
    value, max_s = bench.job_throughput(4.0, 8)
    assert (value, max_s) == (2.0, 4.0)
