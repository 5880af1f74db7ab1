"""bench.py's multi-rank aggregation, run as two gloo ranks on the CPU.

With N GPUs the benchmark runs N independent ranks (replicas of one problem, or distinct cells
of an ensemble); the job time is the slowest rank's and the whole-job throughput counts every
rank's own sites."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms_local = [4.0, 6.0][rank]
    value, ms = bench.aggregate_throughput(1_000_000, 10, ms_local)
    uneven, _ = bench.aggregate_throughput([1_000_000, 3_000_000][rank], 10, ms_local)
    out[rank] = (value, ms, bench.reduce_max(rank + 0.5), uneven, bench.reduce_sum(rank + 1.0))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        value, ms, m, uneven, total = out[r]
        assert ms == 6.0
        assert m == 1.5 and total == 3.0
        # 2 replicas x 1e6 sites x 10 steps / 6 ms
        assert abs(value - 2 * 1_000_000 * 10 / 6e-3 / 1e6) < 1e-6
        # ranks with their own cells: (1e6 + 3e6) sites x 10 steps / 6 ms
        assert abs(uneven - 4_000_000 * 10 / 6e-3 / 1e6) < 1e-6


def test_single_process_is_the_identity():
    import bench
    assert bench.reduce_max(3.25) == 3.25
    value, ms = bench.aggregate_throughput(1000, 5, 2.0)
    assert ms == 2.0 and abs(value - 1000 * 5 / 2e-3 / 1e6) < 1e-12
