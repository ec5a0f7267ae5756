"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the job time
is the slowest rank's, and throughput counts every replica's frames."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


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
    ms = 100.0 + 50.0 * rank            # rank 1 is slower
    slow = bench.slowest_rank_ms(ms, world)
    out[rank] = slow
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_and_job_throughput_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == 150.0
    import bench
    # two replicas of 2500 frames, 10 steps, 150 ms in total
    assert bench.job_throughput(2500, 10, 2, 150.0) == pytest.approx(2 * 2500 * 10 / 0.15)
    assert bench.slowest_rank_ms(42.0, 1) == 42.0
