"""The N-GPU bench path on CPU: independent replicas (one per rank), no data-path collective,
a job that ends when its slowest rank does (max over ranks) and a whole-job rate over all
ranks' bytes, exercised with world_size-2 gloo process groups."""
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


def _rank_main(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        own_ms = [40.0, 55.5][rank]                       # rank 1 is the slow replica
        slowest = bench.max_over_ranks(own_ms, dist, "cpu")
        results[rank] = (slowest, bench.whole_job_rate(1 << 30, world, slowest))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_time_and_whole_job_rate():
    world = 2
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), results), nprocs=world, join=True)
        got = dict(results)
    assert got[0][0] == got[1][0] == 55.5                # both ranks agree on the slowest time
    rate = got[0][1]
    assert rate == pytest.approx(2 * (1 << 30) / 0.0555 / 1e9)   # all ranks' bytes / that time
    assert got[1][1] == rate


def test_single_rank_rate():
    import bench
    assert bench.whole_job_rate(3 << 30, 1, 1000.0) == pytest.approx(3 * (1 << 30) / 1e9)
