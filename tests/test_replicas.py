"""Host-side multi-GPU logic (replicas only) on CPU with world-size-2 gloo
process groups: view sharding and the throughput combination."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2003_10558_gb300.replicas import combine, shard_views  # noqa: E402


def test_shard_views_partition_and_balance():
    sizes = [512 * 512, 1024 * 1024, 2048 * 1024, 1920 * 1080, 512 * 512, 1024 * 1024, 2048 * 1024]
    for world in (1, 2, 3, 4, 8):
        parts = [shard_views(sizes, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
    with pytest.raises(ValueError):
        shard_views(sizes, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [100, 300, 200, 400, 50]
        mine = shard_views(sizes, rank, world)
        units = sum(sizes[i] for i in mine)
        seconds = 1.0 + rank  # the slower rank decides the time
        total, tmax = combine(units, seconds)
        got = [None] * world
        dist.all_gather_object(got, mine)
        q.put((rank, total, tmax, got))
    finally:
        dist.destroy_process_group()


def test_combine_with_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, tmax, got in res:
        assert total == 1050.0 and tmax == 2.0
        assert sorted(i for part in got for i in part) == [0, 1, 2, 3, 4]


def test_combine_without_group_is_local():
    assert combine(7, 0.5) == (7, 0.5)
