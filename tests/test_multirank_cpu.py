"""The multi-GPU mode of bench.py runs independent replicas (one grid per rank, no
exchange step): timings are reduced with a max over ranks and the whole-job rate counts
every rank's cells.  Checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [10.0 + 5.0 * rank, 3.0 - rank]  # rank 1 is slower in the first timing
    ms_max, e2e_max = bench.max_over_ranks(local, world)
    rate = bench.whole_job_rate(world, 1000, 20, ms_max / 1e3)
    dist.barrier()
    q.put((rank, ms_max, e2e_max, rate))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, e2e_max, rate in res:
        assert ms_max == 15.0 and e2e_max == 3.0
        assert abs(rate - 2 * 1000 * 20 / 0.015 / 1e6) < 1e-9


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 3
    assert bench.run_reference(Args()) == 0
