"""Host logic of the multi-GPU benchmark path on CPU: two gloo ranks, each
timing its own independent cloud; the job time is the max over ranks and the
throughput counts every rank's units (weak scaling, no data-path collective)."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [10.0, 25.0][rank]
    t, value = bench.aggregate(local_ms, 1000, world, dist, "cpu")
    out[rank] = (t, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate_takes_the_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for rank in range(world):
        t, value = res[rank]
        assert t == pytest.approx(25.0)
        assert value == pytest.approx(2 * 1000 / 25e-3)


def test_single_rank_aggregate_is_local():
    import bench
    t, value = bench.aggregate(4.0, 500, 1)
    assert t == 4.0 and value == pytest.approx(500 / 4e-3)
