"""The multi-GPU path of bench.py (independent replicas, barrier, slowest
rank's time) on two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slowest
    ms = bench.max_over_ranks(local_ms, dist, torch.device("cpu"))
    dist.barrier()
    out[rank] = (ms, bench.replica_rate(world, 4096 * 4096, 50, ms), bench.rank_workload(rank).seed)
    dist.destroy_process_group()


def test_two_ranks_report_the_slowest_rank_and_the_whole_job_rate():
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    assert res[0][1] == pytest.approx(2 * 4096 * 4096 * 50 / 0.150)
    assert res[0][2] != res[1][2]           # each rank solves its own seeded problem
