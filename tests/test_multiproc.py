"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Replicas only (the solver runs on one GPU per rank, no data-path collective): what the ranks
share is the barrier and the max-over-ranks timing, and for the serving stream the disjoint
split of requests.  Checked here without a GPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    t = bench.max_over_ranks(1.0 + rank, world)
    mine = bench.shard(10, rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    dist.destroy_process_group()
    q.put((rank, t, got))


def test_two_gloo_ranks_time_and_shard():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, got in out:
        assert t == 2.0                      # max over ranks of 1 + rank
        assert sorted(got[0] + got[1]) == list(range(10))
        assert not set(got[0]) & set(got[1])


def test_single_rank_helpers_need_no_process_group():
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    bench.barrier(1)
