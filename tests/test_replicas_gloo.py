"""The multi-GPU path is replicas only: each rank runs the whole workload and the
benchmark reports the slowest rank's time and the summed work.  Checked here with
two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, cells = bench.aggregate_replicas(10.0 + 5.0 * rank, 1e9 * (rank + 1), torch.device("cpu"), world)
    out[rank] = (ms, cells)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        assert out[r] == (15.0, 3e9)


def test_aggregate_single_rank():
    import torch
    import bench
    assert bench.aggregate_replicas(12.5, 7.0, torch.device("cpu"), 1) == (12.5, 7.0)
