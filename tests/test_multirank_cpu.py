"""Host logic of the multi-rank bench path on CPU: two gloo ranks (127.0.0.1) shard the batched
instances with no overlap and agree on the max-over-ranks step time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.shard(64, rank, world)
        got = [None] * world
        dist.all_gather_object(got, mine)
        t = bench.max_over_ranks(1.5 + rank, dist, device="cpu")
        q.put((rank, got, t))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_shard_and_max_over_ranks_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, t in res:
        flat = [k for part in got for k in part]
        assert sorted(flat) == list(range(64))          # every instance on exactly one rank
        assert max(len(g) for g in got) - min(len(g) for g in got) <= 1
        assert t == 1.5 + (world - 1)                  # every rank sees the slowest rank's time


def test_single_process_needs_no_group():
    import bench
    assert bench.shard(5, 0, 1) == list(range(5))
    assert bench.max_over_ranks(2.0, None) == 2.0
