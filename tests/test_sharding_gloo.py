"""Multi-rank placement of independent systems, run as two gloo ranks on CPU:
every system is owned by exactly one rank, and the ranks' predicted walk
costs are balanced by the longest-processing-time rule (hand-computed cases,
Graham's 4/3 bound, never worse than dealing systems round robin by size)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1811_02761_gb300.sharding import (local_csr, partition_systems, rank_loads,
                                              system_costs)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, sizes, cost, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        offsets = np.concatenate([[0], np.cumsum(sizes)])
        mine = partition_systems(sizes, world, cost)[rank]
        local, idx = local_csr(offsets, mine)
        load = float(np.asarray(cost, float)[mine].sum())
        got = [None] * world
        dist.all_gather_object(got, (mine.tolist(), int(local[-1]), idx.tolist(), load))
        if rank == 0:
            q.put(got)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_partition_two_gloo_ranks(world):
    g = np.random.default_rng(3)
    sizes = g.integers(1024, 65536, 61)
    # walk cost per particle varies by system (as it does between Plummer and
    # Hernquist systems of different N): cost is not proportional to size
    cost = sizes * g.uniform(200.0, 2000.0, sizes.size)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, sizes, cost, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    systems = sorted(s for g in got for s in g[0])
    assert systems == list(range(sizes.size))
    counts = [g[1] for g in got]
    assert sum(counts) == sizes.sum()
    parts = np.concatenate([np.array(g[2]) for g in got])
    assert np.array_equal(np.sort(parts), np.arange(sizes.sum()))
    # each rank's cost share: within the largest system of the mean, and a
    # makespan no worse than round robin by particle count
    loads = np.array([g[3] for g in got])
    assert np.isclose(loads.sum(), cost.sum())
    assert loads.max() - loads.mean() <= cost.max()
    rr = np.argsort(-sizes, kind="stable")
    rr_loads = rank_loads([rr[r::world] for r in range(world)], cost)
    assert loads.max() <= rr_loads.max()


def test_partition_hand_cases():
    # costs 7 5 4 3 3 2 on two ranks, most expensive first onto the least
    # loaded rank: 7->0, 5->1, 4->1 (9), 3->0 (10), 3->1 (12), 2->0 (12)
    parts = partition_systems(np.ones(6), 2, [7, 5, 4, 3, 3, 2])
    assert [p.tolist() for p in parts] == [[0, 3, 5], [1, 2, 4]]
    assert rank_loads(parts, [7, 5, 4, 3, 3, 2]).tolist() == [12.0, 12.0]
    # equal sizes, one expensive system: by size (round robin) the expensive
    # one shares a rank (loads 11, 2); by cost it is alone (10, 3)
    parts = partition_systems([100, 100, 100, 100], 2, [10, 1, 1, 1])
    assert [p.tolist() for p in parts] == [[0], [1, 2, 3]]
    assert partition_systems([100, 100, 100, 100], 2)[0].tolist() == [0, 2]
    # without costs the size is the cost
    assert [p.tolist() for p in partition_systems([5, 9, 1], 2)] == [[1], [0, 2]]
    with pytest.raises(ValueError):
        partition_systems([1, 2], 2, [1.0])
    with pytest.raises(ValueError):
        partition_systems([1, 2], 2, [1.0, -1.0])


@pytest.mark.parametrize("world", [2, 3])
def test_partition_within_graham_bound(world):
    """LPT's makespan is at most (4/3 - 1/(3m)) times the optimum, found here
    by brute force over every assignment of a few systems; any list schedule
    also stays within the mean load plus (1 - 1/m) times the largest cost."""
    import itertools
    g = np.random.default_rng(world)
    for _ in range(30):
        k = int(g.integers(1, 8))
        cost = g.lognormal(0.0, 1.5, k)
        loads = rank_loads(partition_systems(np.ones(k), world, cost), cost)
        opt = min(np.bincount(np.array(a, dtype=np.int64), weights=cost, minlength=world).max()
                  for a in itertools.product(range(world), repeat=k))
        assert loads.max() <= (4 / 3 - 1 / (3 * world)) * opt * (1 + 1e-12)
        assert loads.max() <= cost.sum() / world + (1 - 1 / world) * cost.max() + 1e-12
        assert np.isclose(loads.sum(), cost.sum())


def test_system_costs_from_groups():
    # three systems [0,4), [4,4) (empty), [4,10); groups in sorted order
    offsets = [0, 4, 4, 10]
    first, count, entries = [0, 2, 4, 7], [2, 2, 3, 3], [10, 20, 5, 1]
    assert system_costs(offsets, first, count, entries).tolist() == [60.0, 0.0, 18.0]
    with pytest.raises(ValueError):
        system_costs(offsets, [10], [1], [1])


def test_local_csr_packs_systems():
    offsets = np.array([0, 3, 3, 10, 12])
    local, idx = local_csr(offsets, [2, 0])
    assert local.tolist() == [0, 7, 10]
    assert idx.tolist() == [3, 4, 5, 6, 7, 8, 9, 0, 1, 2]
