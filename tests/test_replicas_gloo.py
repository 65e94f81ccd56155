"""Host logic of the N > 1 benchmark path (independent replicas) on CPU ranks
over gloo: max-over-ranks timing, whole-job value, distinct replica seeds, and
the reference arm running on rank 0 only."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = 100.0 + 50.0 * rank
        ms_max = bench.reduce_max(local_ms, "cpu")
        value = bench.replica_value(world, 10, ms_max)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(rank))

        class Args:
            steps, warmup = 1, 0
        ref = bench.run_reference(Args, rank, world) if rank != 0 else "skipped"
        out[rank] = (ms_max, value, seeds, ref)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_aggregation_gloo(world):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    res = dict(out)
    slowest = 100.0 + 50.0 * (world - 1)
    for r in range(world):
        ms_max, value, seeds, ref = res[r]
        assert ms_max == slowest
        assert value == pytest.approx(world * 10 / (slowest / 1000.0))
        assert len(set(seeds)) == world
    assert res[1][3] is None          # only rank 0 runs the reference arm


def test_reduce_max_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.reduce_max(3.5, "cpu") == 3.5
    assert bench.replica_value(1, 4, 2000.0) == 2.0
