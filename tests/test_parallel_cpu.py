"""The multi-rank path on CPU: two gloo ranks shard a point set, each
evaluates its shard (with the oracle: no GPU here), and the gathered shards
equal the unsharded result; the timing reduction takes the maximum."""
import os
import socket

import numpy as np
import pytest

from paper_2510_05282_b300.parallel import shard_range


def test_shard_range_covers_exactly():
    for n in (0, 1, 7, 100, 65_600):
        for world in (1, 2, 3, 8):
            spans = [shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    from paper_2510_05282_b300 import inputs
    from paper_2510_05282_b300.parallel import max_over_ranks, shard_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pts = inputs.random_sphere_points(1000, stream="tests")
        a, b = shard_range(pts.shape[0], rank, world)
        part = oracle.real_sh(pts[a:b], 9, nthreads=1)
        gathered = [None] * world
        dist.all_gather_object(gathered, part)
        t = max_over_ranks(1.5 + rank)
        if rank == 0:
            q.put((np.concatenate(gathered), t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_gather(oracle_mod):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    full, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_2510_05282_b300 import inputs
    pts = inputs.random_sphere_points(1000, stream="tests")
    assert np.array_equal(full, oracle_mod.real_sh(pts, 9, nthreads=1))
    assert t == 2.5
