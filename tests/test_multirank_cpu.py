"""The benchmark's multi-rank aggregation on two gloo ranks (CPU): each rank
decodes its own shard, the job's step time is the slowest rank's, and the
throughput counts every rank's bits (no collective touches decoded data)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total_ms = [100.0, 140.0][rank]  # rank 1 is slower
    ms, value = bench.aggregate(total_ms, 10, 1_000_000, world, "cpu")
    q.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in res:
        assert ms == pytest.approx(14.0)  # the slowest rank, per step
        assert value == pytest.approx(2 * 1_000_000 / 14.0e-3 / 1e6)


def test_single_rank_is_plain_throughput():
    import bench
    ms, value = bench.aggregate(50.0, 5, 2_000_000, 1, "cpu")
    assert ms == 10.0 and value == pytest.approx(200.0)
