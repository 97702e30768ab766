"""The benchmark's multi-rank plumbing on CPU: two gloo ranks, each with its
own timing, agree on the slowest rank's time (the whole-job value is the
pixels of all ranks over that time), and the barrier returns on both."""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    ws, r, local = bench.dist_setup()
    bench.barrier(ws)
    t = bench.max_over_ranks(1.0 + rank, ws)  # rank 1 is the slowest
    q.put((r, local, ws, t))
    bench.barrier(ws)
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=100) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 0, 2, 2.0), (1, 1, 2, 2.0)]
