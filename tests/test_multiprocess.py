"""The N > 1 path of bench.py on CPU: world-size-2 gloo process groups check
the max-over-ranks timing and the sharding of independent instances (no
data-path collective; ranks only agree on the slowest time)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [12.5, 30.0][rank]
    t = bench.max_over_ranks(local, dist)
    lo, hi = bench.shard_units(64, rank, world)
    dist.barrier()
    q.put((rank, t, lo, hi))
    dist.destroy_process_group()


def test_max_over_ranks_and_instance_shards_with_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [30.0, 30.0]          # both ranks see the slowest time
    shards = [(r[2], r[3]) for r in res]
    assert shards == [(0, 32), (32, 64)]


def test_shards_cover_uneven_counts_exactly_once():
    import bench
    for n in (1, 7, 64, 65):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = bench.shard_units(n, r, world)
                seen += list(range(lo, hi))
            assert seen == list(range(n))
