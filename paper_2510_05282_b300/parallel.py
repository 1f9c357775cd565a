"""Multi-GPU helpers.  The evaluation shards without an exchange step: points,
projector atoms and serving requests are independent, so each rank (or each
GPU of one process) works on its own part and nothing crosses GPUs on the
data path.  This module holds the host-side logic of that split:

* shard_range: contiguous point ranges (plain evaluation, strong scaling);
* partition_atoms / sub_problem / scatter_values: projector atoms dealt to
  ranks by cost, sum over a rank's atoms of n_a (lmax_a + 1)^2 values (the
  work of an atom is proportional to the values it writes), each rank's atoms
  forming a problem of their own whose values land back in the global CSR
  layout by atom;
* assign_requests and Dispatcher: serving requests dealt to one server per
  GPU by outstanding cost, completions collected from every server;
* max_over_ranks: the timing reduction of the benchmark.
"""
from __future__ import annotations

import dataclasses
import heapq

import numpy as np


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [start, stop) of n items for `rank` of `world`; the first
    n % world ranks get one extra item."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over the ranks of the default process group (the
    value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- projectors

def atom_costs(prob) -> np.ndarray:
    """Values each atom writes, n_a (lmax_a + 1)^2: the work of its rows."""
    n = np.diff(np.asarray(prob.point_offsets, dtype=np.int64))
    lm = np.asarray(prob.species_lmax)[np.asarray(prob.atom_species)].astype(np.int64)
    return n * (lm + 1) ** 2


def _lpt(costs: np.ndarray, world: int) -> list[np.ndarray]:
    """Longest-processing-time-first assignment: items in decreasing cost,
    each to the currently least loaded part (ties to the lowest part index;
    equal costs in index order, so the result is deterministic).  Each part's
    items are returned in increasing index order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, dtype=np.int64)
    order = np.lexsort((np.arange(costs.size), -costs))
    heap = [(0, r) for r in range(world)]
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(i))
        heapq.heappush(heap, (load + int(costs[i]), r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def partition_atoms(prob, world: int) -> list[np.ndarray]:
    """Atoms of a projector problem dealt to `world` ranks by cost (sum of
    n_a (lmax_a + 1)^2), largest first to the least loaded rank.  The largest
    rank load exceeds the mean by at most one atom's cost."""
    return _lpt(atom_costs(prob), world)


def sub_problem(prob, atoms: np.ndarray):
    """The projector problem of the atoms `atoms` alone (in that order): the
    same grid, species and radial tables, the atoms' positions and sphere
    lists, and output offsets re-based to a CSR of its own."""
    atoms = np.asarray(atoms, dtype=np.int64)
    poff = np.asarray(prob.point_offsets, dtype=np.int64)
    pidx = np.asarray(prob.point_index)
    n = poff[atoms + 1] - poff[atoms]
    lists = [pidx[poff[a]:poff[a + 1]] for a in atoms]
    new_poff = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
    lm = np.asarray(prob.species_lmax)[np.asarray(prob.atom_species)[atoms]].astype(np.int64)
    new_ooff = np.concatenate([[0], np.cumsum(n * (lm + 1) ** 2)]).astype(np.int64)
    return dataclasses.replace(
        prob, atom_pos=np.ascontiguousarray(np.asarray(prob.atom_pos)[atoms]),
        atom_species=np.ascontiguousarray(np.asarray(prob.atom_species)[atoms]),
        atom_rc=np.ascontiguousarray(np.asarray(prob.atom_rc)[atoms]),
        point_offsets=new_poff,
        point_index=(np.concatenate(lists) if lists else pidx[:0]).astype(pidx.dtype),
        out_offsets=new_ooff)


def scatter_values(prob, atoms: np.ndarray, values: np.ndarray, out: np.ndarray) -> None:
    """Writes the values of sub_problem(prob, atoms) into their places in the
    global output `out` (CSR by atom, prob.out_offsets)."""
    ooff = np.asarray(prob.out_offsets, dtype=np.int64)
    pos = 0
    for a in np.asarray(atoms, dtype=np.int64):
        m = int(ooff[a + 1] - ooff[a])
        out[ooff[a]:ooff[a + 1]] = values[pos:pos + m]
        pos += m
    if pos != values.shape[0]:
        raise ValueError("values do not match the atoms' blocks")


# --------------------------------------------------------------------------- serving

def request_cost(n: int, lmax: int, fp64: bool) -> int:
    """Bytes a request writes, n (lmax + 1)^2 x element size: the work of its
    rows (the evaluator is bound by its output or, for binary64 rows, by
    FP64 instructions, both proportional to the values)."""
    return int(n) * (int(lmax) + 1) ** 2 * (8 if fp64 else 4)


def assign_requests(costs, world: int) -> list[np.ndarray]:
    """A batch of requests dealt to `world` servers by cost (the LPT rule of
    partition_atoms)."""
    return _lpt(np.asarray(costs, dtype=np.int64), world)


class Dispatcher:
    """One serving front end over several servers (one per GPU, each a
    shm_serve server or anything with the same submit / wait_any / release
    methods).  Each request goes to the server with the least outstanding
    cost (submitted, not yet collected); a server that answers busy is
    skipped for the next least loaded one.  Tickets are (server index,
    server ticket).  The servers share nothing: a request's rows are computed
    on one GPU, as shm_eval would compute them there."""

    def __init__(self, servers):
        if not servers:
            raise ValueError("no servers")
        self.servers = list(servers)
        self.load = [0] * len(self.servers)
        self.cost: dict[tuple[int, int], int] = {}
        self._next = 0

    def submit(self, n: int, lmax: int, dtype, fp64: bool, **kw):
        """Returns (server, ticket), or None when every server is busy."""
        c = request_cost(n, lmax, fp64)
        for s in sorted(range(len(self.servers)), key=lambda i: (self.load[i], i)):
            t = self.servers[s].submit(n, lmax, dtype, **kw)
            if t is not None:
                self.load[s] += c
                self.cost[(s, t)] = c
                return s, t
        return None

    def wait_any(self, timeout_ms: int = 0):
        """(status, (server, ticket), result) of a completed request from any
        server (servers polled round robin from the one after the last hit);
        status 5 (time-out) when none has one within about timeout_ms."""
        import time
        deadline = time.monotonic() + max(timeout_ms, 0) / 1e3
        k = len(self.servers)
        while True:
            for j in range(k):
                s = (self._next + j) % k
                st, t, r = self.servers[s].wait_any(timeout_ms=0)
                if st != 5:
                    self._next = (s + 1) % k
                    return st, (s, t), r
            if time.monotonic() >= deadline:
                return 5, None, None
            time.sleep(50e-6)

    def release(self, key) -> None:
        s, t = key
        self.servers[s].release(t)
        self.load[s] -= self.cost.pop((s, t), 0)
