"""Placement of independent systems on ranks (one process per GPU).

Independent systems need no exchange, so a multi-GPU run gives each rank
whole systems and runs no collective on the data path.  Systems are placed by
their predicted walk cost with the longest-processing-time rule: most
expensive first, each onto the rank with the least cost so far.  Its makespan
is at most (4/3 - 1/(3 world)) times the best possible (Graham 1969).  The
cost of a system is what its groups' interaction counts add up to in a walk
(system_costs); without costs the particle count stands in for it.
"""
from __future__ import annotations

import numpy as np


def partition_systems(sizes, world: int, cost=None):
    """Return, for each rank, the sorted indices of the systems it owns.

    sizes: particles per system; cost (optional): predicted walk cost per
    system (e.g. its interactions in the last walk).  Ties go to the lower
    rank, so every rank computes the same placement without communicating."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    w = sizes.astype(np.float64) if cost is None else np.asarray(cost, dtype=np.float64)
    if w.shape != sizes.shape:
        raise ValueError("cost must have one entry per system")
    if np.any(w < 0) or not np.all(np.isfinite(w)):
        raise ValueError("costs must be finite and >= 0")
    order = np.argsort(-w, kind="stable")
    load = np.zeros(world)
    owner = np.empty(sizes.size, dtype=np.int64)
    for s in order:
        r = int(np.argmin(load))  # first minimum: the lowest rank among equals
        owner[s] = r
        load[r] += w[s]
    return [np.flatnonzero(owner == r) for r in range(world)]


def rank_loads(parts, cost):
    """Summed cost of each rank's systems."""
    cost = np.asarray(cost, dtype=np.float64)
    return np.array([cost[np.asarray(p, dtype=np.int64)].sum() for p in parts])


def system_costs(offsets, grp_first, grp_count, grp_entries):
    """Interactions of each system in a walk of the forest: the sum over its
    groups of list entries x members.  Groups are given in the forest's
    (sorted) particle order, where every system occupies the same index range
    [offsets[s], offsets[s+1]) as in the caller's CSR layout."""
    offsets = np.asarray(offsets, dtype=np.int64)
    first = np.asarray(grp_first, dtype=np.int64)
    inter = np.asarray(grp_entries, dtype=np.float64) * np.asarray(grp_count, dtype=np.float64)
    sys_of = np.searchsorted(offsets, first, side="right") - 1
    if first.size and (sys_of.min() < 0 or sys_of.max() >= offsets.size - 1):
        raise ValueError("a group starts outside the systems' index range")
    return np.bincount(sys_of, weights=inter, minlength=offsets.size - 1)


def local_csr(offsets, systems):
    """CSR offsets of the given systems packed back to back, and the index
    map from packed particles to the global arrays."""
    offsets = np.asarray(offsets, dtype=np.int64)
    sizes = offsets[np.asarray(systems) + 1] - offsets[np.asarray(systems)]
    local = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    idx = (np.concatenate([np.arange(offsets[s], offsets[s + 1]) for s in systems])
           if len(systems) else np.zeros(0, np.int64))
    return local, idx
