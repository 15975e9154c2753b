"""Replica bookkeeping across processes (world size 2, gloo on the CPU)."""

import os
import socket

import pytest

from paper_2604_16118_gb300 import replicas


def test_shard_covers_units_once():
    for n in (0, 1, 5, 128, 131):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                b, e = replicas.shard(n, r, world)
                assert 0 <= b <= e <= n
                seen.extend(range(b, e))
            assert seen == list(range(n))
            sizes = [replicas.shard(n, r, world)[1] - replicas.shard(n, r, world)[0] for r in range(world)]
            assert max(sizes) - min(sizes) <= 1


def test_shard_rejects_bad_rank():
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)
    with pytest.raises(ValueError):
        replicas.shard(-1, 0, 1)


def test_single_process_passthrough():
    assert replicas.reduce_timing(3.5, 7.0) == (3.5, 7.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank times a different share: rank r ran (r + 1) units in 10 (r + 1) ms
        ms, work = replicas.reduce_timing(10.0 * (rank + 1), float(rank + 1), dist, "cpu")
        b, e = replicas.shard(7, rank, world)
        q.put((rank, ms, work, b, e))
    finally:
        dist.destroy_process_group()


def test_reduce_timing_gloo_world2():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, work, b, e in res:
        assert ms == 20.0            # the slowest rank's time
        assert work == 3.0           # 1 + 2 units
    assert [(b, e) for _, _, _, b, e in res] == [(0, 4), (4, 7)]
