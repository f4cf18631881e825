"""The replica path of bench.py on two CPU ranks (gloo): every rank gets the
slowest rank's time and the whole-job rate counts all ranks' units."""
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
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    assert bench.env_rank() == (rank, rank, world)
    dist.barrier()
    ms = 10.0 * (rank + 1)                    # rank 1 is the slower one
    m = bench.max_over_ranks(ms, torch.device("cpu"))
    out[rank] = (m, bench.whole_job_rate(1000.0, world, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_rate():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert out[0] == out[1]
    m, rate = out[0]
    assert m == 20.0
    assert rate == pytest.approx(1000.0 * 2 / 0.020)
