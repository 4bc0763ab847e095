"""Multi-process path on CPU: two gloo ranks (127.0.0.1) exercise the
sharding, timing and gather helpers the bench uses under torchrun."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_0812_2976_gb300 import dist as kdist


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_covers_exactly_once():
    for n in (0, 1, 5, 4096, 1 << 20):
        for world in (1, 2, 3, 8):
            spans = [kdist.shard(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        kdist.shard(10, 2, 2)


def test_shard_by_work_balances():
    rng = np.random.default_rng(0)
    work = rng.integers(16, 1025, 5000) * rng.integers(1, 7, 5000)
    parts = kdist.shard_by_work(work, 4)
    allidx = np.sort(np.concatenate(parts))
    assert np.array_equal(allidx, np.arange(work.size))
    loads = [work[p].sum() for p in parts]
    assert max(loads) / min(loads) < 1.01


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = kdist.env()
        n = 11
        a, b = kdist.shard(n, r, w)
        local = torch.arange(a, b, dtype=torch.float64) * 2.0
        counts = [kdist.shard(n, i, w)[1] - kdist.shard(n, i, w)[0] for i in range(w)]
        full = kdist.gather_shards(local, counts)
        slowest = kdist.max_over_ranks(0.5 + r)
        q.put((r, full.tolist(), slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, full, slowest in out:
        assert full == [2.0 * i for i in range(11)]
        assert slowest == 1.5
