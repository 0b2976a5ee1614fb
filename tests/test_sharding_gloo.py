"""Multi-rank placement of independent systems, run as two gloo ranks on CPU:
every system is owned by exactly one rank, and the ranks' particle counts are
balanced to within the largest system."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1811_02761_gb300.sharding import local_csr, partition_systems


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, sizes, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        offsets = np.concatenate([[0], np.cumsum(sizes)])
        mine = partition_systems(sizes, world)[rank]
        local, idx = local_csr(offsets, mine)
        got = [None] * world
        dist.all_gather_object(got, (mine.tolist(), int(local[-1]), idx.tolist()))
        if rank == 0:
            q.put(got)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_partition_two_gloo_ranks(world):
    sizes = np.random.default_rng(3).integers(1024, 65536, 61)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, sizes, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    systems = sorted(s for g in got for s in g[0])
    assert systems == list(range(sizes.size))
    counts = [g[1] for g in got]
    assert max(counts) - min(counts) <= sizes.max()
    parts = np.concatenate([np.array(g[2]) for g in got])
    assert np.array_equal(np.sort(parts), np.arange(sizes.sum()))


def test_local_csr_packs_systems():
    offsets = np.array([0, 3, 3, 10, 12])
    local, idx = local_csr(offsets, [2, 0])
    assert local.tolist() == [0, 7, 10]
    assert idx.tolist() == [3, 4, 5, 6, 7, 8, 9, 0, 1, 2]
