"""The multi-GPU path is replicas only (each rank runs the whole workload on
its own GPU, no data-path collective); its host logic -- the max-over-ranks
step time and the whole-job throughput -- runs here as two gloo ranks."""
import os
import socket

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, value, qps = bench.combine_ranks(10.0 + 5.0 * rank, 1_000_000, 20, world, dist)
    out[rank] = (ms, value, qps)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    # the manager's server process is spawned too: earlier tests leave this
    # process multi-threaded, and a fork of it may deadlock
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, value, qps = res[rank]
        assert ms == 15.0  # the slowest rank sets the step time
        assert value == 1_000_000 * 2 / 0.015
        assert qps == 20 * 2 / 0.015


def test_single_rank_needs_no_collective():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(20.0, 100, 4, 1) == (20.0, 100 / 0.02, 4 / 0.02)
