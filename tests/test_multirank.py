"""Host logic of the multi-GPU (replica) benchmark on CPU: two gloo ranks
reduce their timed regions to the slowest one, and the whole-job MLUPS
counts the cells of every rank."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = [12.5, 20.0][rank]
    out[rank] = bench.max_over_ranks(ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_reduction_and_aggregate():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 20.0
    import bench

    assert bench.aggregate_mlups(262144, 100, 2, 20.0) == pytest.approx(2 * 262144 * 100 / 0.02 / 1e6)


def test_single_process_max_is_identity():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
