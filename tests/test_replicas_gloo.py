"""The N > 1 path of bench.py runs independent replicas: the job's time is the
slowest rank's and its work the sum of all ranks'.  Checked with two gloo
ranks on the CPU (no GPU, no collective on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_info() == (world, rank, rank)
        local_ms = [100.0, 160.0][rank]
        units = [3.0e12, 5.0e12][rank]
        ms, total = bench.aggregate_over_ranks(local_ms, units, dist, "cpu")
        out[rank] = (ms, total)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_max_time_and_sum_work():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        ms, total = out[r]
        assert ms == 160.0 and total == 8.0e12
    # the throughput the JSON line reports: 8e12 flop in 0.16 s
    assert abs(8.0e12 / 0.160 / 1e12 - 50.0) < 1e-9


def test_single_process_aggregate_is_local():
    import bench
    assert bench.aggregate_over_ranks(12.5, 7.0) == (12.5, 7.0)
