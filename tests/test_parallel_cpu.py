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


# ---------------------------------------------------------------- projectors and serving split

def _small_projector_problem():
    from paper_2510_05282_b300 import inputs
    return inputs.projector_problem(n_atoms=9, box=6.0, h=0.25, rc_range=(1.0, 2.2), n_species=3,
                                    lmax_choices=(2, 3, 4), n_rad=200, r_min=1e-3, r_max=3.0, extra=21)


def test_partition_atoms_by_cost_is_balanced_and_complete():
    from paper_2510_05282_b300.parallel import atom_costs, partition_atoms
    prob = _small_projector_problem()
    cost = atom_costs(prob)
    for world in (1, 2, 3, 4):
        parts = partition_atoms(prob, world)
        assert sorted(np.concatenate(parts).tolist()) == list(range(prob.n_atoms))
        loads = [int(cost[p].sum()) for p in parts]
        assert max(loads) - cost.sum() / world <= cost.max()      # the LPT bound
    # the same partition every time (ties broken by index)
    assert all(np.array_equal(a, b) for a, b in zip(partition_atoms(prob, 3), partition_atoms(prob, 3)))


def test_sub_problems_rebuild_the_global_output(oracle_mod):
    from paper_2510_05282_b300.parallel import partition_atoms, scatter_values, sub_problem
    prob = _small_projector_problem()
    full = oracle_mod.projectors(prob, nthreads=1)
    out = np.full_like(full, np.nan)
    for atoms in partition_atoms(prob, 3):
        sub = sub_problem(prob, atoms)
        assert sub.n_values == sum(int(prob.out_offsets[a + 1] - prob.out_offsets[a]) for a in atoms)
        scatter_values(prob, atoms, oracle_mod.projectors(sub, nthreads=1), out)
    assert np.array_equal(out, full)


def _proj_worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    from paper_2510_05282_b300.parallel import partition_atoms, scatter_values, sub_problem
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = _small_projector_problem()                 # every rank builds the same seeded problem
        atoms = partition_atoms(prob, world)[rank]
        vals = oracle.projectors(sub_problem(prob, atoms), nthreads=1)
        gathered = [None] * world
        dist.all_gather_object(gathered, (atoms, vals))
        if rank == 0:
            out = np.full(prob.n_values, np.nan)
            for a, v in gathered:
                scatter_values(prob, a, v, out)
            q.put(out)
    finally:
        dist.destroy_process_group()


def _serve_worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    from paper_2510_05282_b300 import inputs
    from paper_2510_05282_b300.parallel import assign_requests, request_cost
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        reqs = inputs.serving_requests(400.0, 0.05, n_lo=50, n_hi=3000)
        costs = [request_cost(r.n, r.lmax, r.dtype == "f64") for r in reqs]
        mine = assign_requests(costs, world)[rank]
        rows = {int(i): oracle.real_sh(inputs.counter_points(reqs[i].seed, reqs[i].n), reqs[i].lmax, nthreads=1)
                for i in mine}
        gathered = [None] * world
        dist.all_gather_object(gathered, rows)
        if rank == 0:
            merged = {}
            for g in gathered:
                assert not set(g) & set(merged)
                merged.update(g)
            q.put((len(reqs), merged))
    finally:
        dist.destroy_process_group()


def _run_two(target):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def test_two_gloo_ranks_partition_projector_atoms(oracle_mod):
    """Two ranks take the atoms partition_atoms deals them, each computes its
    sub-problem (the oracle here: no GPU), and the gathered values, put back
    by atom, equal the unsharded problem's."""
    out = _run_two(_proj_worker)
    assert np.array_equal(out, oracle_mod.projectors(_small_projector_problem(), nthreads=1))


def test_two_gloo_ranks_split_serving_requests(oracle_mod):
    """Two ranks (one server each in a real run) take the requests
    assign_requests deals them; every request is served exactly once and its
    rows equal the unsharded evaluation."""
    from paper_2510_05282_b300 import inputs
    n, merged = _run_two(_serve_worker)
    reqs = inputs.serving_requests(400.0, 0.05, n_lo=50, n_hi=3000)
    assert n == len(reqs) and sorted(merged) == list(range(n))
    for i, r in enumerate(reqs):
        assert np.array_equal(merged[i], oracle_mod.real_sh(inputs.counter_points(r.seed, r.n), r.lmax, nthreads=1))


class _FakeServer:
    """A stand-in with the Server interface: completes a request on the
    first wait_any after it was submitted; refuses beyond `capacity`."""

    def __init__(self, capacity=1000):
        self.capacity, self.pending, self.next, self.released = capacity, [], 1, []

    def submit(self, n, lmax, dtype, **kw):
        if len(self.pending) >= self.capacity:
            return None
        t = self.next
        self.next += 1
        self.pending.append((t, n, lmax))
        return t

    def wait_any(self, timeout_ms=0):
        if not self.pending:
            return 5, 0, None
        t, n, lmax = self.pending.pop(0)
        return 0, t, (n, lmax)

    def release(self, t):
        self.released.append(t)


def test_dispatcher_routes_by_outstanding_cost():
    from paper_2510_05282_b300.parallel import Dispatcher, request_cost
    srv = [_FakeServer(), _FakeServer(capacity=1)]
    d = Dispatcher(srv)
    k1 = d.submit(1_000_000, 9, "f64", fp64=True)        # both idle: server 0
    k2 = d.submit(10, 0, "f32", fp64=False)              # server 1 is the less loaded
    k3 = d.submit(10, 0, "f32", fp64=False)              # server 1 is full: server 0 takes it
    assert k1[0] == 0 and k2[0] == 1 and k3[0] == 0
    assert d.load == [request_cost(1_000_000, 9, True) + request_cost(10, 0, False), request_cost(10, 0, False)]
    got = []
    while True:
        st, key, r = d.wait_any(timeout_ms=0)
        if st == 5:
            break
        got.append(key)
        d.release(key)
    assert sorted(got) == sorted([k1, k2, k3]) and d.load == [0, 0]
    srv[1].capacity = 0
    srv[0].capacity = 0
    assert d.submit(5, 1, "f32", fp64=False) is None
