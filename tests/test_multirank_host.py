"""The multi-GPU path of bench.py is independent replicas: its only cross-rank
logic is host-side (barrier, slowest rank's time, summed work). Exercised here with
two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r = bench.Ranks(dist, "cpu")
    r.barrier()
    # rank 0: 200 ms per step and 1000 points; rank 1: 250 ms and 3000 points
    ms, value = bench.aggregate(r, 200.0 + 50.0 * rank, 1000 + 2000 * rank)
    out[rank] = (ms, value, bench.dist_setup(None))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_replicas():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for rank in range(world):
        ms, value, (w, rk, local) = out[rank]
        assert ms == 250.0                      # the slowest replica sets the time
        assert value == pytest.approx(4000 / 0.25)   # all ranks' points over that time
        assert (w, rk, local) == (world, rank, rank)


def test_single_process_needs_no_collective():
    import bench

    ms, value = bench.aggregate(bench.Ranks(None), 500.0, 1000)
    assert ms == 500.0 and value == 2000.0
