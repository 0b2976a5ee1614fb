"""Placement of independent systems on ranks (one process per GPU).

Independent systems need no exchange, so a multi-GPU run gives each rank
whole systems and runs no collective on the data path.  Systems are dealt
largest first, round robin, which keeps the per-rank particle counts within
one system of each other.
"""
from __future__ import annotations

import numpy as np


def partition_systems(sizes, world: int):
    """Return, for each rank, the sorted indices of the systems it owns."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = np.argsort(-sizes, kind="stable")
    return [np.sort(order[r::world]) for r in range(world)]


def local_csr(offsets, systems):
    """CSR offsets of the given systems packed back to back, and the index
    map from packed particles to the global arrays."""
    offsets = np.asarray(offsets, dtype=np.int64)
    sizes = offsets[np.asarray(systems) + 1] - offsets[np.asarray(systems)]
    local = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    idx = (np.concatenate([np.arange(offsets[s], offsets[s + 1]) for s in systems])
           if len(systems) else np.zeros(0, np.int64))
    return local, idx
